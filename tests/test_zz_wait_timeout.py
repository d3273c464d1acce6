"""Failure detection without a fault: a device wait that nothing completes
gives up after its bounded number of polls, the context's error word carries
FHEON_ERR_TIMEOUT to the next fheon_sync (once), and the context goes on
computing bit-exact results.  No GPU is faulted, trapped or hung: the wait
is cut to 1024 polls."""
import numpy as np
import pytest

import gpu_common
from oracle import ckks
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_and_the_context_goes_on():
    pr = gpu_common.Pair("small_n12", rot_steps=[3])
    g, F = pr.g, pr.F
    g.sync()
    g.selftest_wait(1024)
    with pytest.raises(F.FheonError) as e:
        g.sync()
    assert e.value.code == -6
    g.sync()                                   # reported once, then cleared
    m = synth.small_int_poly(pr.P["seed"], 21, pr.N, 1 << 30)
    ct, oct_ = pr.encrypt_both(m, nonce=21, level=4)
    y = g.rotate(ct, 3)
    want = pr.o.rotate(oct_, g.galois_elt(3), pr.okeys[g.galois_elt(3)])
    assert gpu_common.mismatch(g.ct_download(y), want) == 0
    with pytest.raises(F.FheonError) as e:
        g.selftest_wait(0)
    assert e.value.code == -1
