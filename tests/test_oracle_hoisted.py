"""Pins of the oracle's hoisted rotations (one raising of c1 shared by several
Galois elements; Halevi-Shoup hoisting in the hybrid key-switching form).

Exact pins: with g = 1, and for any g when c1 is a constant polynomial (sigma_g
fixes it, and the coefficient-wise ModUp of a constant is a constant), raising
commutes with sigma_g, so the hoisted result must equal the plain rotation bit
for bit.  Semantic pins: decryption is sigma_g of the message up to the
key-switching noise; for a generic c1 the residues differ from the plain
rotation (the fast base conversion is not odd), which detects a raising taken
after the automorphism instead of before it."""
import numpy as np
import pytest

from oracle import ckks
from paper_2510_03996_gb300 import synth


@pytest.fixture(scope="module")
def tiny():
    P = synth.params("tiny")
    N = 1 << P["logN"]
    mods = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    L = len(P["qbits"])
    ctx = ckks.Ctx(N, mods[:L], mods[L:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    return ctx, P, se, pk


def _centered(v, m):
    v = int(v) % m
    return v - m if v > m // 2 else v


def _ct(ctx, pk, seed, nonce, level):
    m = synth.small_int_poly(seed, nonce & 0xFF, ctx.N, 1 << 30)
    return ctx.drop_level(ctx.encrypt(pk, m, nonce), level)


@pytest.mark.parametrize("level", [4, 3, 1])
def test_identity_element_equals_plain_rotation(tiny, level):
    ctx, P, se, pk = tiny
    key = ctx.rotkey(se, 1)
    ct = _ct(ctx, pk, 31, 3, level)
    got = ctx.rotate_hoisted(ct, [1], [key])[0]
    assert np.array_equal(got, ctx.rotate(ct, 1, key))


@pytest.mark.parametrize("level", [4, 2])
def test_constant_c1_equals_plain_rotation_for_every_g(tiny, level):
    ctx, P, se, pk = tiny
    N = ctx.N
    ct = _ct(ctx, pk, 32, 4, level).copy()
    # c1 := NTT of the constant polynomial c (per limb), c0 left generic
    rng = np.random.default_rng(5)
    for i, q in enumerate(ctx.q[:level]):
        coeffs = np.zeros(N, dtype=np.uint64)
        coeffs[0] = int(rng.integers(0, q))
        ct[1, i] = ckks.ntt(coeffs, q, ctx.psi[i])
    gs = [ckks.galois_elt(r, N) for r in (1, 3, -1, 7)] + [2 * N - 1]
    keys = [ctx.rotkey(se, g) for g in gs]
    got = ctx.rotate_hoisted(ct, gs, keys)
    for r, (g, k) in enumerate(zip(gs, keys)):
        assert np.array_equal(got[r], ctx.rotate(ct, g, k)), g


def test_decrypts_to_automorphism_and_differs_from_plain(tiny):
    """decrypt(hoisted(ct, g)) = sigma_g(decrypt(ct)) + key-switching noise (the
    bound of the plain rotation's pin); the residues are not the plain
    rotation's, and the two decryptions differ by noise only."""
    ctx, P, se, pk = tiny
    N = ctx.N
    steps = [1, 3, -1, 7]
    gs = [ckks.galois_elt(r, N) for r in steps]
    keys = [ctx.rotkey(se, g) for g in gs]
    bound = 4 * (ctx.K + 1) * (N + 1) + 64
    for level in (4, 2):
        ct = _ct(ctx, pk, 33, 40 + level, level)
        q0 = ctx.q[0]
        dec0 = ctx.decrypt_coeffs(se, ct)
        hs = ctx.rotate_hoisted(ct, gs, keys)
        for g, k, h in zip(gs, keys, hs):
            want = ckks.automorph_coeff(np.array([v % q0 for v in dec0], dtype=np.uint64), q0, g)
            dec = ctx.decrypt_coeffs(se, h)
            assert max(abs(_centered(a - int(b), q0)) for a, b in zip(dec, want)) <= bound
            plain = ctx.rotate(ct, g, k)
            assert not np.array_equal(h, plain)
            dp = ctx.decrypt_coeffs(se, plain)
            assert max(abs(_centered(a - b, q0)) for a, b in zip(dec, dp)) <= 2 * bound


def test_each_rotation_is_independent_of_the_others(tiny):
    ctx, P, se, pk = tiny
    N = ctx.N
    gs = [ckks.galois_elt(r, N) for r in (2, -3, 5)]
    keys = [ctx.rotkey(se, g) for g in gs]
    ct = _ct(ctx, pk, 34, 9, 3)
    together = ctx.rotate_hoisted(ct, gs, keys)
    for r, (g, k) in enumerate(zip(gs, keys)):
        assert np.array_equal(together[r], ctx.rotate_hoisted(ct, [g], [k])[0])
    assert ctx.rotate_hoisted(ct, [], []).shape == (0, 2, 3, N)


def test_hoisted_rotation_moves_slots():
    """decode(decrypt(hoisted(enc(encode z), 5^r))) = roll(z, -r) within noise."""
    P = synth.params("small_n12")
    N = 1 << P["logN"]
    mods = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    L = len(P["qbits"])
    ctx = ckks.Ctx(N, mods[:L], mods[L:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    z = synth.uniform_slots(7, 1, N // 2, complex_=True)
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z, N, P["scale"]), 2), 3)
    steps = (1, 5, -2, 28)
    gs = [ckks.galois_elt(r, N) for r in steps]
    outs = ctx.rotate_hoisted(ct, gs, [ctx.rotkey(se, g) for g in gs])
    for r, o in zip(steps, outs):
        assert np.max(np.abs(ctx.decode_ct(se, o, P["scale"]) - np.roll(z, -r))) < 1e-6
