"""fheon_rotate_noalloc: the rotation for callers that must not allocate device
memory while they rotate (a pre-partitioned serving process, a path that
cannot pay for cudaMalloc/cudaFree, work inside a stream capture).  It uses
the library's fixed scratch array instead of the allocator and must give
exactly what fheon_rotate gives.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

import gpu_common


@pytest.fixture(scope="module")
def pair():
    # N = 2^13, L = 3, K = 1: a rotation needs 31 limbs x 64 KiB = 2 MiB of scratch
    return gpu_common.Pair("conv_n13", rot_steps=[1, -28, 57])


def test_noalloc_rotation_matches_rotate_twice(pair):
    g = pair.g
    out = g.ct_create(pair.L, pair.P["scale"])  # made once, before the calls
    cases = [(3, 1), (2, -28)]  # two calls in a row, different levels and steps
    for i, (level, step) in enumerate(cases):
        m = synth.small_int_poly(40, i, pair.N, 1 << 40)
        ct, _ = pair.encrypt_both(m, nonce=500 + i, level=level)
        want = g.ct_download(g.rotate(ct, step))
        g.rotate_noalloc(ct, step, out)
        got = g.ct_download(out)
        assert g.ct_info(out)[0] == level
        # integer work: the tolerance is zero
        assert got.shape == want.shape and np.array_equal(got, want)


def test_noalloc_rejects_what_it_cannot_do(pair):
    g, F = pair.g, pair.F
    m = synth.small_int_poly(41, 0, pair.N, 1 << 20)
    ct, _ = pair.encrypt_both(m, nonce=600)
    small_out = g.ct_create(1)
    with pytest.raises(F.FheonError) as e:  # output too small: it would need an allocation
        g.rotate_noalloc(ct, 1, small_out)
    assert e.value.code == -1
    with pytest.raises(F.FheonError) as e:  # no key
        g.rotate_noalloc(ct, 2, g.ct_create(pair.L))
    assert e.value.code == -3


def test_noalloc_rejects_sizes_beyond_the_array():
    import torch
    from paper_2510_03996_gb300 import fheon as F
    F.use_torch_allocator()
    P = synth.params("rot_n16")
    ctx = F.Context(1 << 16, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                    stream=torch.cuda.current_stream().cuda_stream)
    ct = ctx.ct_create(24, P["scale"])
    with pytest.raises(F.FheonError) as e:  # level 24 needs 176 MiB of scratch, the array holds 32 MiB
        ctx.rotate_noalloc(ct, 1, ctx.ct_create(24))
    assert e.value.code == -1 and "scratch" in str(e.value)
