"""The C-ABI library builds, loads without a GPU, and exports every function
include/fheon.h declares (no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fheon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fheon_[a-z0-9_]+)\s*\(", src)) - {"fheon_alloc_fn", "fheon_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_2510_03996_gb300 import build as B
    B.build()
    from paper_2510_03996_gb300 import fheon as F
    return F


def test_library_exports_every_declared_symbol(lib):
    lib.load()
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    declared = _declared()
    assert len(declared) >= 40
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    # the binding marshals every declared call under the same name
    assert sorted(set(declared) - set(lib.exported_symbols())) == []


def test_error_strings_without_gpu(lib):
    L = lib.load()
    assert L.fheon_error_string(0) == b"ok"
    assert L.fheon_error_string(-3) == b"rotation key missing"
    # argument errors are reported before any device work
    assert L.fheon_ctx_create_bits(1000, None, 0, None, 0, 1, 1.0, 0, None, None) == -1
