"""Failure injection on the host: an allocator hook that refuses every block
makes the calls that need memory fail with FHEON_ERR_OOM and a message;
blocks made before go back through the hook that made them; with the
caching allocator back, the same context rotates to the same bits."""
import pytest

import gpu_common
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


def test_refusing_allocator_reports_oom_and_the_context_goes_on():
    pr = gpu_common.Pair("small_n12", rot_steps=[1])
    g, F = pr.g, pr.F
    m = synth.small_int_poly(22, 0, pr.N, 1 << 40)
    ct, _ = pr.encrypt_both(m, nonce=22)
    want = g.ct_download(g.rotate(ct, 1))
    asked = []

    def refuse(nbytes, stream, user):
        asked.append(int(nbytes))
        return None

    def free(ptr, nbytes, stream, user):  # nothing is ever allocated through it
        pass

    F.set_allocator(refuse, free)
    try:
        with pytest.raises(F.FheonError) as e:
            g.ct_create(3)
        assert e.value.code == -2 and "allocation" in str(e.value)
        with pytest.raises(F.FheonError) as e:
            g.rotate(ct, 1)
        assert e.value.code == -2
        assert asked and all(n > 0 for n in asked)
    finally:
        F.use_torch_allocator()
    assert gpu_common.mismatch(g.ct_download(g.rotate(ct, 1)), want) == 0
