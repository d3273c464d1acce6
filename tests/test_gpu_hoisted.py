"""Hoisted rotations on the GPU against the oracle's hoisted rotations: whole
ciphertexts, bit-exact, at every level of a 5-limb chain (partial last digits),
in every key-switching schedule, grouped in batches, and at the batched
rotation workload's full size."""
import numpy as np
import pytest

import gpu_common
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

STEPS = [1, -1, 5, 100, 2047]


@pytest.fixture(scope="module")
def small():
    # N = 2^12, Q = 5 limbs, P = 2 limbs, dnum = 3 -> alpha = 2, beta = 3
    return gpu_common.Pair("small_n12", rot_steps=STEPS)


def _want(pr, oct_, steps):
    gs = [pr.g.galois_elt(r) for r in steps]
    return pr.o.rotate_hoisted(oct_, gs, [pr.okeys[g] for g in gs])


@pytest.mark.parametrize("level", [5, 4, 3, 2, 1])
def test_hoisted_bit_exact(small, level):
    m = synth.small_int_poly(21, level, small.N, 1 << 40)
    ct, oct_ = small.encrypt_both(m, nonce=3000 + level, level=level)
    outs = small.g.rotate_hoisted(ct, STEPS)
    want = _want(small, oct_, STEPS)
    for o, w in zip(outs, want):
        assert gpu_common.mismatch(small.g.ct_download(o), w) == 0
    # one rotation alone is still hoisted (raised before the automorphism)
    one = small.g.rotate_hoisted(ct, [STEPS[2]])[0]
    assert gpu_common.mismatch(small.g.ct_download(one), want[2]) == 0


@pytest.mark.parametrize("schedule", [0, 1, 2, 3, 4, 5, 6, 7, 9, 11, 13, 15, 17, 25, 31])
def test_hoisted_every_schedule(small, schedule):
    g = small.g
    old = g.get_schedule()
    g.set_schedule(schedule)
    try:
        m = synth.small_int_poly(22, schedule, small.N, 1 << 40)
        ct, oct_ = small.encrypt_both(m, nonce=3100 + schedule, level=5)
        outs = g.rotate_hoisted(ct, STEPS)
        for o, w in zip(outs, _want(small, oct_, STEPS)):
            assert gpu_common.mismatch(g.ct_download(o), w) == 0
    finally:
        g.set_schedule(old)


def test_batch_hoisted_groups(small):
    """Items sharing an input share one raising; inputs at different levels,
    items interleaved; a plain batch of the same items keeps its own bits."""
    g = small.g
    a, oa = small.encrypt_both(synth.small_int_poly(23, 0, small.N, 1 << 40), nonce=3200, level=5)
    b, ob = small.encrypt_both(synth.small_int_poly(23, 1, small.N, 1 << 40), nonce=3201, level=3)
    plan = [(a, 1), (b, 5), (a, -1), (b, 100), (a, 2047), (b, 1)]
    ins = [c for c, _ in plan]
    steps = [s for _, s in plan]
    outs = [g.ct_create(1) for _ in plan]
    g.rotate_batch_hoisted(ins, outs, steps)
    wa = dict(zip([1, -1, 2047], _want(small, oa, [1, -1, 2047])))
    wb = dict(zip([5, 100, 1], _want(small, ob, [5, 100, 1])))
    for (c, s), o in zip(plan, outs):
        w = wa[s] if c is a else wb[s]
        assert gpu_common.mismatch(g.ct_download(o), w) == 0
    # the plain batch of the same items: the non-hoisted oracle rotation
    g.rotate_batch(ins, outs, steps)
    for (c, s), o in zip(plan, outs):
        gg = g.galois_elt(s)
        w = small.o.rotate(oa if c is a else ob, gg, small.okeys[gg])
        assert gpu_common.mismatch(g.ct_download(o), w) == 0


def test_hoisted_errors(small):
    g = small.g
    F = small.F
    ct, _ = small.encrypt_both(synth.small_int_poly(24, 0, small.N, 1 << 40), nonce=3300, level=4)
    with pytest.raises(F.FheonError) as e:
        g.rotate_hoisted(ct, [1, 3])  # no key for step 3
    assert e.value.code == -3
    with pytest.raises(F.FheonError) as e:
        g.rotate_hoisted(ct, [1, 5], [ct, g.ct_create(1)])  # output aliases the input
    assert e.value.code == -1
    o = g.ct_create(1)
    with pytest.raises(F.FheonError) as e:
        g.rotate_hoisted(ct, [1, 5], [o, o])  # repeated output
    assert e.value.code == -1
    assert g.rotate_hoisted(ct, []) == []


def test_hoisted_full_size_sampled():
    """Batched-rotation workload parameters (N = 2^16, 24 x 50-bit Q, 4 x 60-bit
    P, dnum 6) at a partial-digit level: two hoisted rotations, whole
    ciphertexts, against the oracle."""
    pr = gpu_common.Pair("rot_n16", rot_steps=[12345, 77])
    m = synth.small_int_poly(25, 0, pr.N, 1 << 40)
    ct, oct_ = pr.encrypt_both(m, nonce=5, level=13)
    outs = pr.g.rotate_hoisted(ct, [12345, 77])
    for o, w in zip(outs, _want(pr, oct_, [12345, 77])):
        assert gpu_common.mismatch(pr.g.ct_download(o), w) == 0
