"""Pins of the oracle's primitives against definitions computed independently
here (pure Python big integers), published test vectors and library routines."""
import os
import random
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import ckks

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brv(x, logn):
    return int(format(x, "0%db" % logn)[::-1], 2) if logn else 0


# ------------------------------------------------------------ ChaCha20
def _read_chacha_golden():
    d = {"out": []}
    for line in open(os.path.join(GOLDEN, "chacha20_rfc8439_2_3_2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        if k == "out":
            d["out"] += [int(x, 16) for x in v]
        elif k == "counter":
            d[k] = int(v[0])
        else:
            d[k] = [int(x, 16) for x in v]
    return d


def test_chacha20_rfc8439_vector():
    g = _read_chacha_golden()
    out = ckks.chacha20_block(g["key"], g["counter"], g["nonce"])
    assert [int(x) for x in out] == g["out"]


def test_chacha20_matches_cryptography_library():
    crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms
    rnd = random.Random(5)
    for _ in range(8):
        key = bytes(rnd.randrange(256) for _ in range(32))
        nonce = bytes(rnd.randrange(256) for _ in range(12))
        ctr = rnd.randrange(1 << 20)
        full_nonce = ctr.to_bytes(4, "little") + nonce
        ks = Cipher(algorithms.ChaCha20(key, full_nonce), mode=None).encryptor().update(bytes(64))
        kw = np.frombuffer(key, dtype="<u4")
        nw = np.frombuffer(nonce, dtype="<u4")
        out = ckks.chacha20_block(kw, ctr, nw)
        assert out.astype("<u4").tobytes() == ks


def test_draw64_is_word_pair_of_block():
    seed, dom, idx = 0x1234_5678_9ABC_DEF0, 7, (3 << 32) | 11
    key = [seed & 0xFFFFFFFF, seed >> 32, 0, 0, 0, 0, 0, 0]
    nonce = [dom, idx & 0xFFFFFFFF, idx >> 32]
    for n in [0, 1, 7, 8, 9, 100, 4097]:
        blk = ckks.chacha20_block(key, n // 8, nonce)
        p = n % 8
        assert ckks.draw64(seed, dom, idx, n) == int(blk[2 * p]) | (int(blk[2 * p + 1]) << 32)


# ------------------------------------------------------------ primes, roots
def test_is_prime_against_sympy():
    sympy = pytest.importorskip("sympy")
    rnd = random.Random(1)
    cases = [2, 3, 4, 561, 1105, 3215031751, 2152302898747, 3474749660383, 341550071728321,
             (1 << 61) - 1, (1 << 62) - 57, 18446744073709551557]
    cases += [rnd.randrange(1 << 62) | 1 for _ in range(300)]
    for n in cases:
        assert ckks.is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("logN,bits", [(13, [60, 40, 40, 60]), (16, [50] * 6 + [60] * 2), (6, [50, 40, 40, 40, 58, 58])])
def test_gen_primes_are_the_largest_ntt_primes(logN, bits):
    sympy = pytest.importorskip("sympy")
    N = 1 << logN
    ps = ckks.gen_primes(N, bits)
    assert len(set(ps)) == len(ps)
    for t, (q, b) in enumerate(zip(ps, bits)):
        assert q % (2 * N) == 1 and q.bit_length() == b and sympy.isprime(q)
        # no larger unused candidate of that size is prime
        c = q + 2 * N
        while c < (1 << b):
            assert (c in ps[:t]) or not sympy.isprime(c)
            c += 2 * N


@pytest.mark.parametrize("q,N", [(17, 8), (97, 16), (7681, 256), (12289, 1024)])
def test_min_psi_brute_force(q, N):
    roots = [x for x in range(1, q) if pow(x, 2 * N, q) == 1 and pow(x, N, q) == q - 1]
    assert ckks.min_psi(q, N) == min(roots)


def test_min_psi_large_prime_properties():
    N = 1 << 13
    q = ckks.gen_primes(N, [60])[0]
    psi = ckks.min_psi(q, N)
    assert pow(psi, N, q) == q - 1
    # psi is the minimum over the odd powers of any primitive root of order 2N
    sq = psi * psi % q
    cur = psi
    for _ in range(N - 1):
        cur = cur * sq % q
        assert cur > psi


# ------------------------------------------------------------ NTT
def _ntt_python(a, q, psi):
    N = len(a)
    logn = N.bit_length() - 1
    return [sum(int(a[i]) * pow(psi, (2 * brv(j, logn) + 1) * i, q) for i in range(N)) % q for j in range(N)]


@pytest.mark.parametrize("q,N", [(17, 8), (97, 16), (7681, 32)])
def test_ntt_definition_brute_force(q, N):
    psi = ckks.min_psi(q, N)
    rnd = random.Random(q)
    a = [rnd.randrange(q) for _ in range(N)]
    assert [int(x) for x in ckks.ntt_def(a, q, psi)] == _ntt_python(a, q, psi)
    assert [int(x) for x in ckks.ntt(a, q, psi)] == _ntt_python(a, q, psi)


def test_ntt_definition_large_prime():
    N = 16
    q = ckks.gen_primes(N, [60])[0]
    psi = ckks.min_psi(q, N)
    a = [random.Random(3).randrange(q) for _ in range(N)]
    assert [int(x) for x in ckks.ntt_def(a, q, psi)] == _ntt_python(a, q, psi)


@pytest.mark.parametrize("logN", [3, 6, 9, 10])
def test_fast_ntt_equals_definition(logN):
    N = 1 << logN
    for bits in (50, 60):
        q = ckks.gen_primes(N, [bits])[0]
        psi = ckks.min_psi(q, N)
        a = np.array([random.Random(logN + bits).randrange(q) for _ in range(N)], dtype=np.uint64)
        A = ckks.ntt(a, q, psi)
        assert np.array_equal(A, ckks.ntt_def(a, q, psi))
        assert np.array_equal(ckks.intt(A, q, psi), a)
        assert np.array_equal(ckks.intt_def(A, q, psi), a)


def _negacyclic_python(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                out[i + j] += int(a[i]) * int(b[j])
            else:
                out[i + j - N] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


def test_convolution_theorem():
    N = 64
    q = ckks.gen_primes(N, [59])[0]
    psi = ckks.min_psi(q, N)
    rnd = random.Random(9)
    a = np.array([rnd.randrange(q) for _ in range(N)], dtype=np.uint64)
    b = np.array([rnd.randrange(q) for _ in range(N)], dtype=np.uint64)
    ab = ckks.negacyclic_mul(a, b, q)
    assert [int(x) for x in ab] == _negacyclic_python(a, b, q)
    lhs = ckks.ntt(ab, q, psi)
    A, B = ckks.ntt(a, q, psi), ckks.ntt(b, q, psi)
    rhs = [int(x) * int(y) % q for x, y in zip(A, B)]
    assert [int(x) for x in lhs] == rhs


# ------------------------------------------------------------ automorphism
def test_automorph_coeff_definition_and_composition():
    N = 32
    q = ckks.gen_primes(N, [40])[0]
    rnd = random.Random(2)
    a = np.array([rnd.randrange(q) for _ in range(N)], dtype=np.uint64)
    for g in [5, 25, 2 * N - 1, 3, 17]:
        out = ckks.automorph_coeff(a, q, g)
        ref = [0] * N
        for i in range(N):
            e = i * g % (2 * N)
            if e < N:
                ref[e] = int(a[i])
            else:
                ref[e - N] = (-int(a[i])) % q
        assert [int(x) for x in out] == ref
    for g, h in [(5, 25), (5, 2 * N - 1), (125, 3)]:
        lhs = ckks.automorph_coeff(ckks.automorph_coeff(a, q, h), q, g)
        assert np.array_equal(lhs, ckks.automorph_coeff(a, q, g * h % (2 * N)))


def test_automorph_is_permutation_in_eval_domain():
    """sigma_g in the bit-reversed evaluation domain permutes values: index j takes
    index j' with 2 brv(j')+1 = (2 brv(j)+1) g mod 2N."""
    N = 64
    logn = 6
    q = ckks.gen_primes(N, [50])[0]
    psi = ckks.min_psi(q, N)
    rnd = random.Random(4)
    a = np.array([rnd.randrange(q) for _ in range(N)], dtype=np.uint64)
    A = ckks.ntt(a, q, psi)
    inv = {2 * brv(j, logn) + 1: j for j in range(N)}
    for g in [5, 25, 5 ** 7 % (2 * N), 2 * N - 1]:
        S = ckks.ntt(ckks.automorph_coeff(a, q, g), q, psi)
        for j in range(N):
            jp = inv[(2 * brv(j, logn) + 1) * g % (2 * N)]
            assert S[j] == A[jp]


# ------------------------------------------------------------ base conversion
def test_bconv_against_exact_crt():
    N = 16
    mods = ckks.gen_primes(N, [50, 50, 50, 60, 60, 40])
    frm, to = mods[:3], mods[3:]
    rnd = random.Random(7)
    D = frm[0] * frm[1] * frm[2]
    xs = [rnd.randrange(D) for _ in range(N)]
    xin = np.array([[x % d for x in xs] for d in frm], dtype=np.uint64)
    out = ckks.bconv(xin, frm, to)
    for k, x in enumerate(xs):
        for t, m in enumerate(to):
            y = int(out[t, k])
            # y = x + u*D mod m for one u in [0, len(frm))
            assert any((x + u * D) % m == y for u in range(len(frm)))


# ------------------------------------------------------------ Gaussian table
def test_cdt_table_against_high_precision():
    getcontext().prec = 60
    sigma, tail = Decimal("3.2"), 20
    rho = [(-(Decimal(k * k)) / (2 * sigma * sigma)).exp() for k in range(-tail, tail + 1)]
    S = sum(rho)
    T = ckks.cdt_table(3.2, tail)
    c = Decimal(0)
    for i, k in enumerate(range(-tail, tail)):
        c += rho[i]
        exact = c / S * (Decimal(2) ** 64)
        # binary64 exp, a 41-term sum and a division: a few dozen ulps at most;
        # a wrong formula (sigma vs sigma^2, a lost factor 2) is off by far more
        assert abs(Decimal(int(T[i])) - exact) <= exact * Decimal(2) ** -45 + 1
    assert all(int(T[i]) < int(T[i + 1]) for i in range(2 * tail - 1))


def test_samplers_statistics():
    N = 1 << 16
    e = ckks.sample_gauss(11, 3, 0, N)
    assert abs(e.mean()) < 0.05 and abs(e.std() - 3.2) < 0.05 and np.abs(e).max() <= 20
    s = ckks.sample_ternary(11, 1, 0, N)
    assert set(np.unique(s)) == {-1, 0, 1}
    counts = np.bincount(s + 1)
    assert np.all(np.abs(counts / N - 1 / 3) < 0.01)
    q = ckks.gen_primes(1 << 13, [50])[0]
    u = ckks.sample_uniform(11, 2, 0, 4096, q)
    assert int(u.max()) < q and abs(float(u.astype(np.float64).mean()) / q - 0.5) < 0.02
    # draws are exactly the documented function of the stream
    lo, hi = ckks.draw64(11, 2, 0, 0), ckks.draw64(11, 2, 0, 1)
    assert int(u[0]) == ((hi << 64) | lo) % q
    assert int(s[5]) == ckks.draw64(11, 1, 0, 5) % 3 - 1
