"""Pins of the oracle's ciphertext product with relinearisation and of its
scalar operations, against exact big-integer arithmetic (schoolbook negacyclic
products, CRT), the relinearisation key's defining relation, and slot-wise
products under decode."""
import numpy as np
import pytest

from oracle import ckks
from paper_2510_03996_gb300 import synth


def _ctx(name):
    P = synth.params(name)
    N = 1 << P["logN"]
    mods = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    L = len(P["qbits"])
    return ckks.Ctx(N, mods[:L], mods[L:], P["dnum"], P["seed"]), P


@pytest.fixture(scope="module")
def tiny():
    ctx, P = _ctx("tiny")
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    return ctx, P, s, se, pk


def _negacyclic(a, b):
    N = len(a)
    out = [0] * N
    for i in range(N):
        if a[i]:
            for j in range(N):
                if i + j < N:
                    out[i + j] += a[i] * b[j]
                else:
                    out[i + j - N] -= a[i] * b[j]
    return out


def _centered(v, Q):
    v %= Q
    return v - Q if v > Q // 2 else v


def _Q(ctx, level):
    Q = 1
    for q in ctx.q[:level]:
        Q *= q
    return Q


def test_relin_key_relation(tiny):
    """b_j + a_j s = e_j + P [limb in digit j] s^2 with |e_j| <= 20 (the CDT tail)."""
    ctx, P, s, se, pk = tiny
    rlk = ctx.relinkey(se)
    N, L = ctx.N, ctx.L
    s2 = _negacyclic([int(x) for x in s], [int(x) for x in s])
    Pm = 1
    for p in ctx.p:
        Pm *= p
    for j in range(ctx.beta):
        for i, m in enumerate(ctx.mod):
            b = ckks.intt(rlk[j, 0, i], m, ctx.psi[i])
            a = ckks.intt(rlk[j, 1, i], m, ctx.psi[i])
            a_s = _negacyclic([int(x) for x in a], [int(x) for x in s])
            in_digit = i < L and i // ctx.alpha == j
            for k in range(N):
                e = int(b[k]) + a_s[k] - (Pm * s2[k] if in_digit else 0)
                assert abs(_centered(e, m)) <= 20


@pytest.mark.parametrize("level", [4, 3, 1])
def test_mul_relin_decrypts_to_the_product(tiny, level):
    """decrypt(mul_relin(a, b)) = decrypt(a) * decrypt(b) + key-switching noise,
    the product taken exactly over the integers, negacyclically."""
    ctx, P, s, se, pk = tiny
    rlk = ctx.relinkey(se)
    ma = synth.small_int_poly(41, level, ctx.N, 1 << 12)
    mb = synth.small_int_poly(42, level, ctx.N, 1 << 12)
    a = ctx.drop_level(ctx.encrypt(pk, ma, 50 + level), level)
    b = ctx.drop_level(ctx.encrypt(pk, mb, 60 + level), level)
    Q = _Q(ctx, level)
    da, db = ctx.decrypt_coeffs(se, a), ctx.decrypt_coeffs(se, b)
    want = _negacyclic(list(da), list(db))
    got = ctx.decrypt_coeffs(se, ctx.mul_relin(a, b, rlk))
    Pm = ctx.p[0] * ctx.p[1]
    Dmax = max(ctx.q[0] * ctx.q[1], ctx.q[2] * ctx.q[3])
    beta = (level + ctx.alpha - 1) // ctx.alpha
    bound = beta * ctx.N * ctx.alpha * Dmax * 20 // Pm + (ctx.K + 1) * (ctx.N + 1) + 1
    assert max(abs(_centered(g - w, Q)) for g, w in zip(got, want)) <= bound
    # the tensor is symmetric in its operands, so the product commutes bit for bit
    assert np.array_equal(ctx.mul_relin(a, b, rlk), ctx.mul_relin(b, a, rlk))


def test_mul_int_and_add_int_are_exact(tiny):
    ctx, P, s, se, pk = tiny
    m = synth.small_int_poly(43, 0, ctx.N, 1 << 30)
    ct = ctx.drop_level(ctx.encrypt(pk, m, 70), 3)
    Q = _Q(ctx, 3)
    d = ctx.decrypt_coeffs(se, ct)
    for v in (7, -3, 1 << 40, -(1 << 50)):
        got = ctx.decrypt_coeffs(se, ctx.mul_int(ct, v))
        assert all(_centered(g - v * x, Q) == 0 for g, x in zip(got, d))
        got = ctx.decrypt_coeffs(se, ctx.add_int(ct, v))
        want = list(d)
        want[0] += v
        assert all(_centered(g - w, Q) == 0 for g, w in zip(got, want))


def test_products_in_slots():
    """decode(mul_relin(enc z1, enc z2)) = z1 * z2 at scale D^2, and after a
    rescale at D^2 / q; a constant product rescaled lands on its target scale."""
    ctx, P = _ctx("small_n12")
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    rlk = ctx.relinkey(se)
    N, D = ctx.N, P["scale"]
    z1 = synth.uniform_slots(9, 0, N // 2)
    z2 = synth.uniform_slots(9, 1, N // 2)
    a = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z1, N, D), 1), 4)
    b = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z2, N, D), 2), 4)
    prod = ctx.mul_relin(a, b, rlk)
    assert np.max(np.abs(ctx.decode_ct(se, prod, D * D) - z1 * z2)) < 1e-6
    r = ctx.rescale(prod)
    # rescale rounding: (|s|_1 + 1)/2 per coefficient, times sqrt(N) in a slot,
    # over the new scale D^2 / q_3 ~ 2^35
    tol = (ctx.N + 1) / 2 * np.sqrt(ctx.N) / (D * D / ctx.q[3])
    assert np.max(np.abs(ctx.decode_ct(se, r, D * D / ctx.q[3]) - z1 * z2)) < tol
    for c, target in ((0.37, D), (-2.5, D / 3.0), (1e-3, D)):
        out = ctx.mul_const_rescale(a, c, target, D)
        assert out.shape[1] == 3
        assert np.max(np.abs(ctx.decode_ct(se, out, target) - c * z1)) < 1e-6
    # K is llround(((c * target) * q) / scale) in binary64
    assert abs(ctx.const_factor(4, 0.37, D, D) - 0.37 * ctx.q[3]) <= 1
    assert ctx.const_factor(4, -2.5, D / 3.0, D) == -round(2.5 / 3.0 * ctx.q[3])
