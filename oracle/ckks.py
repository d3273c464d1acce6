"""Python face of the CPU oracle: full-RNS CKKS with hybrid key switching.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library.

Arrays are numpy: polynomials ``uint64[n_limbs][N]`` (limb-major), ciphertexts
``uint64[2][level][N]`` in the evaluation domain, keys over all L+K moduli.
The arithmetic lives in ckks_oracle.c; this module adds only marshalling and
the exact big-integer CRT used by decoding (paper Sec. 3.2 decoding of the
canonical embedding, with the centred lift modulo Q_level).
"""
import numpy as np

from . import _lib
from ._lib import u64p, i64p, u32p, dblp

import ctypes


def _p(a, t):
    return a.ctypes.data_as(t)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# ---------------------------------------------------------------- scalars
def is_prime(n):
    return bool(_lib.lib().oracle_is_prime(int(n)))


def gen_primes(N, bits):
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    out = np.zeros(len(bits), dtype=np.uint64)
    rc = _lib.lib().oracle_gen_primes(N, _p(bits, u32p), len(bits), _p(out, u64p))
    if rc != 0:
        raise ValueError("no prime for bit sizes %s at N=%d" % (list(bits), N))
    return [int(x) for x in out]


def min_psi(q, N):
    return int(_lib.lib().oracle_min_psi(int(q), N))


def llround(x):
    """Round half away from zero (C llround) of a binary64 value."""
    return int(_lib.lib().oracle_llround(float(x)))


def galois_elt(r, N):
    """g = 5^r mod 2N for a slot rotation by r (slot i <- slot i+r); r may be negative."""
    n = N // 2
    return pow(5, r % n, 2 * N)


CONJ = "conj"


# ---------------------------------------------------------------- sampler
def chacha20_block(key_words, counter, nonce_words):
    k = np.ascontiguousarray(key_words, dtype=np.uint32)
    n = np.ascontiguousarray(nonce_words, dtype=np.uint32)
    out = np.zeros(16, dtype=np.uint32)
    _lib.lib().oracle_chacha20_block(_p(k, u32p), counter, _p(n, u32p), _p(out, u32p))
    return out


def draw64(seed, domain, idx, n):
    return int(_lib.lib().oracle_draw64(seed, domain, idx, n))


def cdt_table(sigma=3.2, tail=20):
    T = np.zeros(2 * tail + 1, dtype=np.uint64)
    _lib.lib().oracle_cdt_table(sigma, tail, _p(T, u64p))
    return T


def sample_ternary(seed, domain, idx, N):
    out = np.zeros(N, dtype=np.int64)
    _lib.lib().oracle_sample_ternary(seed, domain, idx, N, _p(out, i64p))
    return out


def sample_gauss(seed, domain, idx, N):
    out = np.zeros(N, dtype=np.int64)
    _lib.lib().oracle_sample_gauss(seed, domain, idx, N, _p(out, i64p))
    return out


def sample_uniform(seed, domain, idx, N, q):
    out = np.zeros(N, dtype=np.uint64)
    _lib.lib().oracle_sample_uniform(seed, domain, idx, N, int(q), _p(out, u64p))
    return out


# ---------------------------------------------------------------- NTT
def _poly_call(fname, a, N, q, psi):
    a = _u64(a)
    out = np.zeros(N, dtype=np.uint64)
    getattr(_lib.lib(), fname)(_p(a, u64p), N, int(q), int(psi), _p(out, u64p))
    return out


def ntt_def(a, q, psi):
    return _poly_call("oracle_ntt_def", a, len(a), q, psi)


def intt_def(a, q, psi):
    return _poly_call("oracle_intt_def", a, len(a), q, psi)


def ntt(a, q, psi):
    return _poly_call("oracle_ntt", a, len(a), q, psi)


def intt(a, q, psi):
    return _poly_call("oracle_intt", a, len(a), q, psi)


def negacyclic_mul(a, b, q):
    a, b = _u64(a), _u64(b)
    out = np.zeros(len(a), dtype=np.uint64)
    _lib.lib().oracle_negacyclic_mul(_p(a, u64p), _p(b, u64p), len(a), int(q), _p(out, u64p))
    return out


def automorph_coeff(a, q, g):
    a = _u64(a)
    out = np.zeros(len(a), dtype=np.uint64)
    _lib.lib().oracle_automorph_coeff(_p(a, u64p), len(a), int(q), int(g), _p(out, u64p))
    return out


def bconv(x, frm, to):
    x = _u64(x)
    frm, to = _u64(frm), _u64(to)
    N = x.shape[1]
    out = np.zeros((len(to), N), dtype=np.uint64)
    _lib.lib().oracle_bconv(_p(x, u64p), _p(frm, u64p), len(frm), _p(to, u64p), len(to), N, _p(out, u64p))
    return out


# ---------------------------------------------------------------- encoding
def encode(z, N, scale):
    """Integer coefficients of round(scale * tau^-1(z)); z complex, len <= N/2."""
    z = np.asarray(z, dtype=np.complex128)
    zr, zi = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
    m = np.zeros(N, dtype=np.int64)
    rc = _lib.lib().oracle_encode(N, _p(zr, dblp), _p(zi, dblp), len(z), float(scale), _p(m, i64p))
    if rc != 0:
        raise OverflowError("encoded coefficient does not fit in 63 bits")
    return m


def decode(m, nslots, scale):
    """Slots of the real polynomial m (float coefficients) divided by scale."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    zr = np.zeros(nslots)
    zi = np.zeros(nslots)
    _lib.lib().oracle_decode(len(m), _p(m, dblp), nslots, float(scale), _p(zr, dblp), _p(zi, dblp))
    return zr + 1j * zi


def crt_centered(residues, moduli):
    """Exact centred CRT lift of limb residues (uint64[l][N]) to Python ints."""
    Q = 1
    for q in moduli:
        Q *= int(q)
    terms = []
    for q in moduli:
        q = int(q)
        Qh = Q // q
        terms.append((Qh * pow(Qh, -1, q), q))
    N = residues.shape[1]
    out = []
    res = [[int(v) for v in row] for row in residues]
    for k in range(N):
        x = 0
        for (c, q), row in zip(terms, res):
            x += row[k] * c
        x %= Q
        if x > Q // 2:
            x -= Q
        out.append(x)
    return out


# ---------------------------------------------------------------- scheme
class Ctx:
    """Oracle scheme context over Q = q_0..q_{L-1}, P = p_0..p_{K-1}."""

    def __init__(self, N, q, p, dnum, seed):
        self.N, self.q, self.p = int(N), [int(x) for x in q], [int(x) for x in p]
        self.L, self.K, self.dnum, self.seed = len(self.q), len(self.p), int(dnum), int(seed)
        qa, pa = _u64(self.q), _u64(self.p)
        self._h = _lib.lib().oracle_ctx_new(self.N, _p(qa, u64p), self.L, _p(pa, u64p), self.K, self.dnum, self.seed)
        self.alpha = _lib.lib().oracle_ctx_alpha(self._h)
        self.beta = _lib.lib().oracle_ctx_beta(self._h)
        self.mod = self.q + self.p
        self.psi = [_lib.lib().oracle_ctx_psi(self._h, i) for i in range(self.L + self.K)]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.lib().oracle_ctx_free(h)
            self._h = None

    # keys
    def keygen_sk(self):
        s = np.zeros(self.N, dtype=np.int64)
        se = np.zeros((self.L + self.K, self.N), dtype=np.uint64)
        _lib.lib().oracle_keygen_sk(self._h, _p(s, i64p), _p(se, u64p))
        return s, se

    def keygen_pk(self, s_eval):
        s_eval = _u64(s_eval)
        pk = np.zeros((2, self.L, self.N), dtype=np.uint64)
        _lib.lib().oracle_keygen_pk(self._h, _p(s_eval, u64p), _p(pk, u64p))
        return pk

    def galois_sk(self, s_eval, g):
        s_eval = _u64(s_eval)
        out = np.zeros_like(s_eval)
        _lib.lib().oracle_galois_sk(self._h, _p(s_eval, u64p), int(g), _p(out, u64p))
        return out

    def keygen_ksk(self, s_eval, sfrom_eval, tag):
        s_eval, sfrom_eval = _u64(s_eval), _u64(sfrom_eval)
        ksk = np.zeros((self.beta, 2, self.L + self.K, self.N), dtype=np.uint64)
        _lib.lib().oracle_keygen_ksk(self._h, _p(s_eval, u64p), _p(sfrom_eval, u64p), int(tag), _p(ksk, u64p))
        return ksk

    def rotkey(self, s_eval, g):
        return self.keygen_ksk(s_eval, self.galois_sk(s_eval, g), g)

    # encryption
    def encrypt(self, pk, m_coeff, nonce):
        pk, m = _u64(pk), _i64(m_coeff)
        ct = np.zeros((2, self.L, self.N), dtype=np.uint64)
        _lib.lib().oracle_encrypt(self._h, _p(pk, u64p), _p(m, i64p), int(nonce), _p(ct, u64p))
        return ct

    def plain_from_coeffs(self, m_coeff, level):
        m = _i64(m_coeff)
        pt = np.zeros((level, self.N), dtype=np.uint64)
        _lib.lib().oracle_plain_from_coeffs(self._h, _p(m, i64p), level, _p(pt, u64p))
        return pt

    def decrypt(self, s_eval, ct):
        ct = _u64(ct)
        level = ct.shape[1]
        s_eval = _u64(s_eval)
        m = np.zeros((level, self.N), dtype=np.uint64)
        _lib.lib().oracle_decrypt(self._h, _p(s_eval, u64p), _p(ct, u64p), level, _p(m, u64p))
        return m

    def to_coeff(self, x, level, with_p=False):
        x = _u64(x)
        out = np.zeros_like(x)
        _lib.lib().oracle_to_coeff(self._h, _p(x, u64p), level, int(with_p), _p(out, u64p))
        return out

    def to_eval(self, x, level, with_p=False):
        x = _u64(x)
        out = np.zeros_like(x)
        _lib.lib().oracle_to_eval(self._h, _p(x, u64p), level, int(with_p), _p(out, u64p))
        return out

    def decrypt_coeffs(self, s_eval, ct):
        """Centred integer message+noise coefficients (Python ints) of ct."""
        m = self.decrypt(s_eval, ct)
        level = m.shape[0]
        return crt_centered(self.to_coeff(m, level), self.q[:level])

    def decode_ct(self, s_eval, ct, scale, nslots=None):
        nslots = nslots or self.N // 2
        coeffs = self.decrypt_coeffs(s_eval, ct)
        return decode(np.array([float(c) for c in coeffs]), nslots, scale)

    # evaluation
    def automorph_eval(self, x, level, g, with_p=False):
        x = _u64(x)
        out = np.zeros_like(x)
        _lib.lib().oracle_automorph_eval(self._h, _p(x, u64p), level, int(with_p), int(g), _p(out, u64p))
        return out

    def modup(self, x_coeff, level, j):
        x = _u64(x_coeff)
        out = np.zeros((level + self.K, self.N), dtype=np.uint64)
        _lib.lib().oracle_modup(self._h, _p(x, u64p), level, j, _p(out, u64p))
        return out

    def moddown(self, x_coeff, level):
        x = _u64(x_coeff)
        out = np.zeros((level, self.N), dtype=np.uint64)
        _lib.lib().oracle_moddown(self._h, _p(x, u64p), level, _p(out, u64p))
        return out

    def keyswitch(self, d_eval, ksk):
        d, k = _u64(d_eval), _u64(ksk)
        level = d.shape[0]
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        _lib.lib().oracle_keyswitch(self._h, _p(d, u64p), level, _p(k, u64p), _p(out, u64p))
        return out

    def rotate(self, ct, g, ksk):
        ct, k = _u64(ct), _u64(ksk)
        level = ct.shape[1]
        out = np.zeros_like(ct)
        _lib.lib().oracle_rotate(self._h, _p(ct, u64p), level, int(g), _p(k, u64p), _p(out, u64p))
        return out

    def relinkey(self, s_eval):
        """Relinearisation key: key-switching key from s^2 to s, tag 0."""
        s_eval = _u64(s_eval)
        sq = np.stack([np.array([(int(x) * int(x)) % m for x in s_eval[i]], dtype=np.uint64)
                       for i, m in enumerate(self.mod)])
        return self.keygen_ksk(s_eval, sq, tag=0)

    def mul_relin(self, a, b, rlk):
        a, b, k = _u64(a), _u64(b), _u64(rlk)
        level = a.shape[1]
        assert b.shape[1] == level
        out = np.zeros_like(a)
        _lib.lib().oracle_mul_relin(self._h, _p(a, u64p), _p(b, u64p), level, _p(k, u64p), _p(out, u64p))
        return out

    def mul_int(self, ct, v):
        ct = _u64(ct)
        out = np.zeros_like(ct)
        _lib.lib().oracle_mul_int(self._h, _p(ct, u64p), ct.shape[1], int(v), _p(out, u64p))
        return out

    def add_int(self, ct, v):
        ct = _u64(ct)
        out = np.zeros_like(ct)
        _lib.lib().oracle_add_int(self._h, _p(ct, u64p), ct.shape[1], int(v), _p(out, u64p))
        return out

    def add_const(self, ct, c, scale):
        """ct + c in every slot: the constant llround(c * scale) added to c0."""
        return self.add_int(ct, llround(float(c) * float(scale)))

    def const_factor(self, level, c, target, scale):
        return int(_lib.lib().oracle_const_factor(self._h, level, float(c), float(target), float(scale)))

    def mul_const_rescale(self, ct, c, target, scale):
        """c * ct rescaled once, landing on scale `target` (ct has scale `scale`)."""
        return self.rescale(self.mul_int(ct, self.const_factor(ct.shape[1], c, target, scale)))

    def rotate_hoisted(self, ct, gs, ksks):
        """Rotations of one ciphertext by each Galois element of `gs`, sharing one
        raising (ModUp + NTT) of c1; ksks[r] is the key of gs[r].  [n][2][level][N]."""
        ct = _u64(ct)
        level = ct.shape[1]
        n = len(gs)
        g = np.array([int(x) for x in gs], dtype=np.uint64)
        k = _u64(np.stack([np.asarray(x, dtype=np.uint64) for x in ksks])) if n else np.zeros(1, np.uint64)
        out = np.zeros((n, 2, level, self.N), dtype=np.uint64)
        if n:
            _lib.lib().oracle_rotate_hoisted(self._h, _p(ct, u64p), level, _p(g, u64p), n, _p(k, u64p), _p(out, u64p))
        return out

    def mul_plain(self, ct, pt):
        ct = _u64(ct)
        level = ct.shape[1]
        pt = _u64(pt[:level])
        out = np.zeros_like(ct)
        _lib.lib().oracle_mul_plain(self._h, _p(ct, u64p), _p(pt, u64p), level, _p(out, u64p))
        return out

    def add(self, x, y):
        x, y = _u64(x), _u64(y)
        if x.shape != y.shape:
            raise ValueError("level mismatch")
        out = np.zeros_like(x)
        _lib.lib().oracle_add(self._h, _p(x, u64p), _p(y, u64p), x.shape[1], _p(out, u64p))
        return out

    def add_plain(self, ct, pt):
        ct = _u64(ct)
        level = ct.shape[1]
        pt = _u64(pt[:level])
        out = np.zeros_like(ct)
        _lib.lib().oracle_add_plain(self._h, _p(ct, u64p), _p(pt, u64p), level, _p(out, u64p))
        return out

    def rescale(self, ct):
        ct = _u64(ct)
        level = ct.shape[1]
        out = np.zeros((2, level - 1, self.N), dtype=np.uint64)
        _lib.lib().oracle_rescale(self._h, _p(ct, u64p), level, _p(out, u64p))
        return out

    def drop_level(self, ct, level):
        return np.ascontiguousarray(ct[:, :level, :])
