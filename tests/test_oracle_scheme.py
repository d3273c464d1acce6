"""Pins of the oracle's scheme steps (keys, encryption, ModUp/ModDown, key
switching, rotation, rescale, plaintext products, encoding) against exact
big-integer arithmetic, schoolbook products and closed-form noise bounds."""
import random

import numpy as np
import pytest

from oracle import ckks
from paper_2510_03996_gb300 import synth


def _ctx(name="tiny"):
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


def _centered(v, m):
    v = int(v) % m
    return v - m if v > m // 2 else v


def _coeff_limbs(ctx, x_eval, level, with_p=False):
    return ctx.to_coeff(x_eval, level, with_p)


def _schoolbook_int(a, b):
    N = len(a)
    out = [0] * N
    for i in range(N):
        if a[i] == 0:
            continue
        for j in range(N):
            if i + j < N:
                out[i + j] += a[i] * b[j]
            else:
                out[i + j - N] -= a[i] * b[j]
    return out


def test_digit_geometry(tiny):
    ctx = tiny[0]
    assert (ctx.alpha, ctx.beta) == (2, 2)


def test_secret_key_is_ternary_and_consistent(tiny):
    ctx, P, s, se, pk = tiny
    assert set(np.unique(s)) <= {-1, 0, 1}
    for i, m in enumerate(ctx.mod):
        coeff = ctx.to_coeff(se[:ctx.L], ctx.L) if i < ctx.L else None
        if coeff is not None:
            assert [_centered(v, m) for v in coeff[i]] == [int(x) for x in s]


def test_public_key_relation(tiny):
    """b + a*s = e with e a small Gaussian polynomial."""
    ctx, P, s, se, pk = tiny
    e_eval = np.stack([((pk[0, i].astype(object) + pk[1, i].astype(object) * se[i].astype(object)) % q)
                       .astype(np.uint64) for i, q in enumerate(ctx.q)])
    e = ctx.to_coeff(e_eval, ctx.L)
    ints = ckks.crt_centered(e, ctx.q)
    assert max(abs(v) for v in ints) <= 20
    for i, q in enumerate(ctx.q):
        assert [_centered(v, q) for v in e[i]] == ints


def test_encrypt_decrypt_noise_bound(tiny):
    ctx, P, s, se, pk = tiny
    m = synth.small_int_poly(1, 0, ctx.N, 1 << 20)
    ct = ctx.encrypt(pk, m, nonce=3)
    dec = ctx.decrypt_coeffs(se, ct)
    err = [d - int(x) for d, x in zip(dec, m)]
    # |v e + e0 + e1 s| <= 20 N + 20 + 20 N  (v, s ternary; |e| <= 20)
    assert max(abs(e) for e in err) <= 40 * ctx.N + 20
    assert max(abs(e) for e in err) > 0


def test_encryption_is_deterministic_per_nonce(tiny):
    ctx, P, s, se, pk = tiny
    m = synth.small_int_poly(1, 1, ctx.N, 100)
    assert np.array_equal(ctx.encrypt(pk, m, 5), ctx.encrypt(pk, m, 5))
    assert not np.array_equal(ctx.encrypt(pk, m, 5), ctx.encrypt(pk, m, 6))


def test_add_and_mul_plain_exact(tiny):
    """decrypt is linear: dec(ct*pt) = dec(ct) * pt and dec(ct+ct') = dec(ct)+dec(ct'),
    exactly, as negacyclic products of the centred integers modulo Q."""
    ctx, P, s, se, pk = tiny
    L = ctx.L
    m1 = synth.small_int_poly(2, 0, ctx.N, 1000)
    m2 = synth.small_int_poly(2, 1, ctx.N, 1000)
    pt_int = synth.small_int_poly(2, 2, ctx.N, 50)
    ct1, ct2 = ctx.encrypt(pk, m1, 10), ctx.encrypt(pk, m2, 11)
    d1, d2 = ctx.decrypt_coeffs(se, ct1), ctx.decrypt_coeffs(se, ct2)
    pt = ctx.plain_from_coeffs(pt_int, L)
    dm = ctx.decrypt_coeffs(se, ctx.mul_plain(ct1, pt))
    assert dm == _schoolbook_int(d1, [int(x) for x in pt_int])
    da = ctx.decrypt_coeffs(se, ctx.add(ct1, ct2))
    assert da == [a + b for a, b in zip(d1, d2)]
    dp = ctx.decrypt_coeffs(se, ctx.add_plain(ct1, pt))
    assert dp == [a + int(b) for a, b in zip(d1, pt_int)]


def test_modup_is_crt_lift_plus_small_multiple(tiny):
    ctx, P, s, se, pk = tiny
    level = 3
    rnd = random.Random(1)
    x = np.array([[rnd.randrange(q) for _ in range(ctx.N)] for q in ctx.q[:level]], dtype=np.uint64)
    for j in range((level + ctx.alpha - 1) // ctx.alpha):
        d0, d1 = j * ctx.alpha, min((j + 1) * ctx.alpha, level)
        D = 1
        for q in ctx.q[d0:d1]:
            D *= q
        xd = ckks.crt_centered(x[d0:d1], ctx.q[d0:d1])
        out = ctx.modup(x, level, j)
        mods = ctx.q[:level] + ctx.p
        for k in range(ctx.N):
            xk = xd[k] % D
            for l, m in enumerate(mods):
                if d0 <= l < d1:
                    assert out[l, k] == x[l, k]
                else:
                    assert any((xk + u * D) % m == int(out[l, k]) for u in range(d1 - d0))


def test_moddown_is_floor_division_minus_small(tiny):
    """ModDown(x) = floor(x / P) - v (mod Q), 0 <= v < K, for x in [0, PQ)."""
    ctx, P, s, se, pk = tiny
    level = 3
    mods = ctx.q[:level] + ctx.p
    Pm = 1
    for p in ctx.p:
        Pm *= p
    QP = Pm
    for q in ctx.q[:level]:
        QP *= q
    rnd = random.Random(2)
    xs = [rnd.randrange(QP) for _ in range(ctx.N)]
    xin = np.array([[x % m for x in xs] for m in mods], dtype=np.uint64)
    out = ctx.moddown(xin, level)
    for k, x in enumerate(xs):
        for i, q in enumerate(ctx.q[:level]):
            assert any((x // Pm - v) % q == int(out[i, k]) for v in range(ctx.K))


def test_rescale_is_floor_division(tiny):
    ctx, P, s, se, pk = tiny
    level = 4
    rnd = random.Random(3)
    Q = 1
    for q in ctx.q[:level]:
        Q *= q
    xs = [rnd.randrange(Q) for _ in range(ctx.N)]
    x_coeff = np.array([[x % q for x in xs] for q in ctx.q[:level]], dtype=np.uint64)
    x_eval = ctx.to_eval(x_coeff, level)
    ct = np.stack([x_eval, x_eval])
    out = ctx.rescale(ct)
    oc = ctx.to_coeff(out[0], level - 1)
    qt = ctx.q[level - 1]
    for k, x in enumerate(xs):
        ref = (x - x % qt) // qt
        for i, q in enumerate(ctx.q[:level - 1]):
            assert int(oc[i, k]) == ref % q


def test_keyswitch_noise_bound(tiny):
    """ks(d) = (b', a') with b' + a' s = d * s_from + e_ks, |e_ks| small."""
    ctx, P, s, se, pk = tiny
    rnd = random.Random(4)
    sfrom_int = [rnd.choice([-1, 0, 1]) for _ in range(ctx.N)]
    sfrom = np.stack([ckks.ntt(np.array([v % m for v in sfrom_int], dtype=np.uint64), m, ctx.psi[i])
                      for i, m in enumerate(ctx.mod)])
    ksk = ctx.keygen_ksk(se, sfrom, tag=0)
    for level in (4, 3, 1):
        d = np.array([[rnd.randrange(q) for _ in range(ctx.N)] for q in ctx.q[:level]], dtype=np.uint64)
        out = ctx.keyswitch(d, ksk)
        dec = ctx.decrypt_coeffs(se, out)
        dint = ckks.crt_centered(ctx.to_coeff(d, level), ctx.q[:level])
        want = _schoolbook_int(dint, sfrom_int)
        Q = 1
        for q in ctx.q[:level]:
            Q *= q
        Pm = ctx.p[0] * ctx.p[1]
        Dmax = max(ctx.q[0] * ctx.q[1], ctx.q[2] * ctx.q[3])  # largest digit modulus
        beta = (level + ctx.alpha - 1) // ctx.alpha
        bound = beta * ctx.N * ctx.alpha * Dmax * 20 // Pm + (ctx.K + 1) * (ctx.N + 1) + 1
        errs = []
        for a, b in zip(dec, want):
            e = (a - b) % Q
            errs.append(e - Q if e > Q // 2 else e)
        assert max(abs(e) for e in errs) <= bound


@pytest.mark.parametrize("r", [1, 3, -1, 7])
def test_rotate_decrypts_to_automorphism(tiny, r):
    """decrypt(rotate(ct, g)) = sigma_g(decrypt(ct)) + small key-switching noise."""
    ctx, P, s, se, pk = tiny
    N = ctx.N
    g = ckks.galois_elt(r, N)
    ksk = ctx.rotkey(se, g)
    m = synth.small_int_poly(5, r & 0xFF, N, 1 << 30)
    ct = ctx.encrypt(pk, m, 20 + (r & 0xFF))
    for level in (4, 2):
        c = ctx.drop_level(ct, level)
        dec0 = ctx.decrypt_coeffs(se, c)
        q0 = ctx.q[0]
        want = ckks.automorph_coeff(np.array([v % q0 for v in dec0], dtype=np.uint64), q0, g)
        rot = ctx.rotate(c, g, ksk)
        dec = ctx.decrypt_coeffs(se, rot)
        err = [_centered(a - int(b), q0) for a, b in zip(dec, want)]
        assert max(abs(e) for e in err) <= 4 * (ctx.K + 1) * (N + 1) + 64


def test_rotate_moves_slots():
    """decode(decrypt(rotate(enc(encode z), 5^r))) = roll(z, -r) within noise."""
    ctx, P = _ctx("small_n12")
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    N, n = ctx.N, ctx.N // 2
    z = synth.uniform_slots(7, 0, n, complex_=True)
    m = ckks.encode(z, N, P["scale"])
    ct = ctx.drop_level(ctx.encrypt(pk, m, 1), 3)
    for r in (1, 5, -2):
        g = ckks.galois_elt(r, N)
        rot = ctx.rotate(ct, g, ctx.rotkey(se, g))
        zz = ctx.decode_ct(se, rot, P["scale"])
        assert np.max(np.abs(zz - np.roll(z, -r))) < 1e-6


def test_conjugation():
    ctx, P = _ctx("small_n12")
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    N = ctx.N
    z = synth.uniform_slots(8, 0, N // 2, complex_=True)
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z, N, P["scale"]), 2), 2)
    g = 2 * N - 1
    rot = ctx.rotate(ct, g, ctx.rotkey(se, g))
    assert np.max(np.abs(ctx.decode_ct(se, rot, P["scale"]) - np.conj(z))) < 1e-6


# ------------------------------------------------------------ encoding
def _decode_fft(m, N, scale):
    """Independent formulation of decoding: u_k = m_k + i m_{k+N/2}, twist by
    zeta^k, length-N/2 DFT with e^{+2 pi i/(N/2)}, slot i = entry (5^i mod 2N - 1)/4."""
    n = N // 2
    m = np.asarray(m, dtype=np.float64)
    u = (m[:n] + 1j * m[n:]) * np.exp(1j * np.pi * np.arange(n) / N)
    V = np.fft.ifft(u) * n  # sum_k u_k e^{+2 pi i a k / n}
    idx = [(pow(5, i, 2 * N) - 1) // 4 for i in range(n)]
    return V[idx] / scale


def test_decode_matches_independent_fft_formulation():
    N = 256
    rnd = np.random.default_rng(0)
    m = rnd.integers(-1000, 1000, N).astype(np.float64)
    assert np.allclose(ckks.decode(m, N // 2, 1.0), _decode_fft(m, N, 1.0), atol=1e-8)


@pytest.mark.parametrize("N", [64, 1024])
def test_encode_decode_roundtrip(N):
    scale = 2.0 ** 30
    z = synth.uniform_slots(3, N, N // 2, complex_=True)
    m = ckks.encode(z, N, scale)
    back = ckks.decode(m.astype(np.float64), N // 2, scale)
    # rounding adds at most 1/2 per coefficient: |error| <= N/2 / scale per slot
    assert np.max(np.abs(back - z)) <= N / 2 / scale


def test_encode_rounds_half_away_from_zero():
    """A constant slot vector z encodes to m_0 = scale * z exactly (every other
    coefficient 0), so the rounding rule shows: half away from zero (2.5 -> 3,
    -2.5 -> -3), to nearest otherwise (2.7 -> 3, 2.4 -> 2, -2.7 -> -3)."""
    N = 64
    for v, want in ((2.5, 3), (-2.5, -3), (2.7, 3), (2.4, 2), (-2.7, -3), (0.5, 1), (-0.5, -1)):
        m = ckks.encode(np.full(N // 2, v), N, 1.0)
        assert int(m[0]) == want and np.all(m[1:] == 0), (v, m[0])


def test_encode_constant_and_partial_slots():
    N = 128
    m = ckks.encode(np.full(N // 2, 0.75), N, 2.0 ** 20)
    assert m[0] == round(0.75 * 2 ** 20) and np.all(m[1:] == 0)
    z = np.array([1.0, -2.0, 0.5])
    m = ckks.encode(z, N, 2.0 ** 30)
    back = ckks.decode(m.astype(np.float64), 3, 2.0 ** 30)
    assert np.max(np.abs(back - z)) < 1e-6


def test_slot_rotation_by_coefficient_automorphism():
    N = 256
    scale = 2.0 ** 30
    z = synth.uniform_slots(4, 0, N // 2, complex_=True)
    m = ckks.encode(z, N, scale)
    q = ckks.gen_primes(N, [62])[0]
    for r in (1, 2, 9, -3):
        g = ckks.galois_elt(r, N)
        mg = ckks.automorph_coeff(np.array([int(v) % q for v in m], dtype=np.uint64), q, g)
        mgi = np.array([_centered(v, q) for v in mg], dtype=np.float64)
        assert np.max(np.abs(ckks.decode(mgi, N // 2, scale) - np.roll(z, -r))) < 1e-6
