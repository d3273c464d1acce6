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


def refusing_allocator(F, asked):
    """Install an allocator hook that refuses (and records) every request."""
    def refuse(nbytes, stream, user):
        asked.append(int(nbytes))
        return None

    def free(ptr, nbytes, stream, user):  # it never hands out a block
        pass
    F.set_allocator(refuse, free)


def test_noalloc_rotation_matches_rotate_twice(pair):
    g, F = pair.g, pair.F
    out = g.ct_create(pair.L, pair.P["scale"])  # made once, before the calls
    cases = [(3, 1), (2, -28)]  # two calls in a row, different levels and steps
    ins, wants = [], []
    for i, (level, step) in enumerate(cases):
        m = synth.small_int_poly(40, i, pair.N, 1 << 40)
        ct, _ = pair.encrypt_both(m, nonce=500 + i, level=level)
        ins.append(ct)
        wants.append(g.ct_download(g.rotate(ct, step)))
    g.sync()
    # with every allocation refused, the rotations still run: they ask for nothing
    asked = []
    refusing_allocator(F, asked)
    try:
        for ct, (level, step), want in zip(ins, cases, wants):
            g.rotate_noalloc(ct, step, out)
            got = g.ct_download(out)
            assert g.ct_info(out)[0] == level
            # integer work: the tolerance is zero
            assert got.shape == want.shape and np.array_equal(got, want)
    finally:
        F.use_torch_allocator()
    assert asked == [], "the allocation-free rotation asked the allocator for %s bytes" % asked


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


def scratch_limbs(l, K, alpha):
    """Workspace limbs of one rotation at level l: xt | ext[beta][l+K] |
    acc[2][l+K] | pc[2][K] | conv[2][l] (the library's layout)."""
    beta = -(-l // alpha)
    return l + beta * (l + K) + 2 * (l + K) + 2 * K + 2 * l


def test_noalloc_limit_at_full_size():
    """N = 2^16, 24 Q primes, K = 4, dnum 6: the 32 MiB array holds level 5
    (59 limbs of 512 KiB, 29.5 MiB), which rotates exactly as fheon_rotate
    does; level 6 (66 limbs, 33 MiB) and level 24 (304 limbs, 152 MiB) are
    refused."""
    pr = gpu_common.Pair("rot_n16", rot_steps=[3])
    g, F = pr.g, pr.F
    limb = pr.N * 8
    assert scratch_limbs(5, pr.g.K, pr.g.alpha) * limb <= 32 << 20 < scratch_limbs(6, pr.g.K, pr.g.alpha) * limb
    assert scratch_limbs(24, pr.g.K, pr.g.alpha) * limb == 152 << 20
    m = synth.small_int_poly(42, 0, pr.N, 1 << 40)
    ct, _ = pr.encrypt_both(m, nonce=700, level=5)
    want = g.ct_download(g.rotate(ct, 3))
    out = g.ct_create(24, pr.P["scale"])
    g.rotate_noalloc(ct, 3, out)
    assert np.array_equal(g.ct_download(out), want)
    for level in (6, 24):
        c = g.ct_create(level, pr.P["scale"])
        with pytest.raises(F.FheonError) as e:
            g.rotate_noalloc(c, 3, out)
        assert e.value.code == -1 and "scratch" in str(e.value)
