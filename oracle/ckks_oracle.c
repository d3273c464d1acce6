/*
 * ckks_oracle.c -- plain, slow CPU oracle of full-RNS CKKS with hybrid key
 * switching, the arithmetic behind FHEON's homomorphic rotation.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; it is written for
 * readability, never for speed: every modular product is a 128-bit product
 * followed by the C `%` operator.
 *
 * What it follows.  FHEON delegates all of CKKS to OpenFHE's RNS-CKKS (paper
 * Sec. 3.2, "Cheon-Kim-Kim-Song (CKKS) Scheme") and names the full-RNS variant
 * of Cheon, Han, Kim, Kim and Song (SAC 2018) and hybrid key switching with
 * "4 digits" (Sec. 6, parameter paragraph).  The paper gives none of the
 * internals; the steps below are the textbook ones:
 *   - negacyclic NTT: evaluation at the odd powers of a 2N-th root psi,
 *     output index j holding a(psi^(2*brv(j)+1)); Cooley-Tukey forward and
 *     Gentleman-Sande inverse butterflies (Longa-Naehrig 2016) for speed at
 *     large N, the O(N^2) definition beside them;
 *   - fast base conversion (Cheon et al. SAC 2018, Sec. 3.2), no correction;
 *   - hybrid key switching (Han-Ki, CT-RSA 2020): digit decomposition,
 *     ModUp, inner product with the key, ModDown;
 *   - floor rescale by the last prime;
 *   - ChaCha20 block function (RFC 8439, Sec. 2.3) as the counter-based
 *     generator every random draw comes from.
 * Conventions the paper leaves open are fixed in the design notes; the ones
 * that change bits are restated at each function below.
 *
 * Layout: a polynomial over moduli m_0..m_{n-1} is u64[n][N], limb-major,
 * residues canonical in [0, m_i).  Ciphertexts are u64[2][level][N] in the
 * evaluation (NTT) domain.  Keys span all L+K moduli: Q limbs first, then P.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* Scalar modular arithmetic: definitions, nothing clever.             */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
static u64 addmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a + b) % m); }
static u64 submod(u64 a, u64 b, u64 m) { return a >= b ? a - b : (u64)(((u128)a + m - b) % m); }
static u64 powmod(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}
/* inverse modulo a prime, by Fermat's little theorem */
static u64 invmod(u64 a, u64 m) { return powmod(a % m, m - 2, m); }
static u64 from_signed(i64 v, u64 m)
{
    if (v >= 0) return (u64)v % m;
    u64 r = (u64)(-(v + 1)) % m; /* -(v+1) avoids overflow at INT64_MIN */
    return (m - 1 - r) % m;
}

static u32 brv(u32 x, u32 logn)
{
    u32 r = 0;
    for (u32 i = 0; i < logn; i++) r |= ((x >> i) & 1u) << (logn - 1 - i);
    return r;
}
static u32 ilog2(u32 n)
{
    u32 l = 0;
    while ((1u << l) < n) l++;
    return l;
}

/* ------------------------------------------------------------------ */
/* Primes and roots of unity.                                          */
/* ------------------------------------------------------------------ */

/* Deterministic Miller-Rabin for 64-bit n (the first twelve prime bases
 * are a known-complete witness set below 3.3e24). */
int oracle_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* For each requested bit size, in order, the largest prime q < 2^bits with
 * q = 1 (mod 2N) not already chosen.  Callers list the Q sizes first and the
 * P sizes after them, so P primes come after Q primes of the same size.
 * Returns 0, or -1 if a size has no such prime of exactly that many bits. */
int oracle_gen_primes(u32 N, const u32 *bits, u32 n, u64 *out)
{
    u64 twoN = 2ull * N;
    for (u32 t = 0; t < n; t++) {
        u32 b = bits[t];
        if (b < 2 || b > 62) return -1;
        u64 top = (1ull << b) - 1;              /* largest b-bit value */
        u64 cand = top - ((top - 1) % twoN);    /* largest <= top with cand = 1 mod 2N */
        u64 lo = 1ull << (b - 1);
        int found = 0;
        for (; cand >= lo && cand > twoN; cand -= twoN) {
            int used = 0;
            for (u32 u = 0; u < t; u++) used |= (out[u] == cand);
            if (!used && oracle_is_prime(cand)) { found = 1; break; }
        }
        if (!found) return -1;
        out[t] = cand;
    }
    return 0;
}

/* The smallest primitive 2N-th root of unity modulo q (q = 1 mod 2N): take
 * psi0 = x^((q-1)/2N) for x = 2, 3, ... until psi0^N = -1, then the minimum
 * over its odd powers, which are exactly the primitive 2N-th roots. */
u64 oracle_min_psi(u64 q, u32 N)
{
    u64 twoN = 2ull * N, psi0 = 0;
    for (u64 x = 2; x < q; x++) {
        psi0 = powmod(x, (q - 1) / twoN, q);
        if (powmod(psi0, N, q) == q - 1) break;
    }
    u64 sq = mulmod(psi0, psi0, q), cur = psi0, best = psi0;
    for (u64 k = 3; k < twoN; k += 2) {
        cur = mulmod(cur, sq, q);
        if (cur < best) best = cur;
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* ChaCha20 (RFC 8439, Sec. 2.3) and the draws built on it.            */
/* ------------------------------------------------------------------ */
static u32 rotl32(u32 v, int c) { return (v << c) | (v >> (32 - c)); }
static void quarter(u32 *x, int a, int b, int c, int d)
{
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 16);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 12);
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 8);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 7);
}
void oracle_chacha20_block(const u32 key[8], u32 counter, const u32 nonce[3], u32 out[16])
{
    u32 s[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                 key[0], key[1], key[2], key[3], key[4], key[5], key[6], key[7],
                 counter, nonce[0], nonce[1], nonce[2]};
    u32 x[16];
    memcpy(x, s, sizeof x);
    for (int r = 0; r < 10; r++) {
        quarter(x, 0, 4, 8, 12); quarter(x, 1, 5, 9, 13);
        quarter(x, 2, 6, 10, 14); quarter(x, 3, 7, 11, 15);
        quarter(x, 0, 5, 10, 15); quarter(x, 1, 6, 11, 12);
        quarter(x, 2, 7, 8, 13); quarter(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

/* Draw number n (64 bits) of the stream (seed, domain, idx): ChaCha20 with
 * key words (seed lo, seed hi, 0 x 6), nonce words (domain, idx lo, idx hi),
 * block counter n/8, and the little-endian word pair 2*(n%8), 2*(n%8)+1. */
u64 oracle_draw64(u64 seed, u32 domain, u64 idx, u64 n)
{
    u32 key[8] = {(u32)seed, (u32)(seed >> 32), 0, 0, 0, 0, 0, 0};
    u32 nonce[3] = {domain, (u32)idx, (u32)(idx >> 32)};
    u32 blk[16];
    oracle_chacha20_block(key, (u32)(n / 8), nonce, blk);
    u32 p = (u32)(n % 8);
    return (u64)blk[2 * p] | ((u64)blk[2 * p + 1] << 32);
}

/* Cumulative table of the discrete Gaussian rho(k) = exp(-k^2/(2 sigma^2))
 * on k = -tail..tail: T[k+tail] = floor(2^64 * sum_{i<=k} rho(i) / sum rho)
 * for k < tail, in binary64 exactly as written (partial sums in increasing
 * k).  A draw u maps to the smallest k with u < T[k+tail], or to tail. */
void oracle_cdt_table(double sigma, int tail, u64 *T)
{
    int n = 2 * tail + 1;
    double *rho = (double *)malloc(sizeof(double) * (size_t)n);
    double S = 0.0;
    for (int k = -tail; k <= tail; k++) {
        rho[k + tail] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        S += rho[k + tail];
    }
    double c = 0.0;
    for (int k = -tail; k < tail; k++) {
        c += rho[k + tail];
        T[k + tail] = (u64)ldexp(c / S, 64);
    }
    T[n - 1] = 0; /* unused */
    free(rho);
}

#define GAUSS_SIGMA 3.2
#define GAUSS_TAIL 20

void oracle_sample_ternary(u64 seed, u32 domain, u64 idx, u32 N, i64 *out)
{
    for (u32 n = 0; n < N; n++) out[n] = (i64)(oracle_draw64(seed, domain, idx, n) % 3) - 1;
}
void oracle_sample_gauss(u64 seed, u32 domain, u64 idx, u32 N, i64 *out)
{
    u64 T[2 * GAUSS_TAIL + 1];
    oracle_cdt_table(GAUSS_SIGMA, GAUSS_TAIL, T);
    for (u32 n = 0; n < N; n++) {
        u64 u = oracle_draw64(seed, domain, idx, n);
        int k = -GAUSS_TAIL;
        while (k < GAUSS_TAIL && u >= T[k + GAUSS_TAIL]) k++;
        out[n] = k;
    }
}
/* uniform residue: the 128-bit draw (hi = draw 2n+1, lo = draw 2n) mod q */
void oracle_sample_uniform(u64 seed, u32 domain, u64 idx, u32 N, u64 q, u64 *out)
{
    for (u32 n = 0; n < N; n++) {
        u64 lo = oracle_draw64(seed, domain, idx, 2ull * n);
        u64 hi = oracle_draw64(seed, domain, idx, 2ull * n + 1);
        out[n] = (u64)((((u128)hi << 64) | lo) % q);
    }
}

/* ------------------------------------------------------------------ */
/* Negacyclic NTT.                                                     */
/* ------------------------------------------------------------------ */

/* Definition: out[j] = sum_i a[i] * psi^((2*brv(j)+1)*i) mod q. O(N^2). */
void oracle_ntt_def(const u64 *a, u32 N, u64 q, u64 psi, u64 *out)
{
    u32 logn = ilog2(N);
    for (u32 j = 0; j < N; j++) {
        u64 w = powmod(psi, 2ull * brv(j, logn) + 1, q), x = 1, acc = 0;
        for (u32 i = 0; i < N; i++) {
            acc = addmod(acc, mulmod(a[i] % q, x, q), q);
            x = mulmod(x, w, q);
        }
        out[j] = acc;
    }
}
/* Definition of the inverse: a[i] = N^-1 sum_j out[j] psi^(-(2*brv(j)+1)*i). */
void oracle_intt_def(const u64 *A, u32 N, u64 q, u64 psi, u64 *out)
{
    u32 logn = ilog2(N);
    u64 pinv = invmod(psi, q), ninv = invmod(N, q);
    for (u32 i = 0; i < N; i++) {
        u64 acc = 0;
        for (u32 j = 0; j < N; j++) {
            u64 e = ((2ull * brv(j, logn) + 1) * i) % (2ull * N);
            acc = addmod(acc, mulmod(A[j] % q, powmod(pinv, e, q), q), q);
        }
        out[i] = mulmod(acc, ninv, q);
    }
}

/* Iterative Cooley-Tukey forward transform, natural-order input, output in
 * the bit-reversed evaluation order above (Longa-Naehrig 2016, Alg. 1). */
static void ntt_fast(u64 *a, u32 N, u64 q, u64 psi)
{
    u32 logn = ilog2(N);
    u64 *tw = (u64 *)malloc(sizeof(u64) * N); /* tw[i] = psi^brv(i) */
    for (u32 i = 0; i < N; i++) tw[i] = powmod(psi, brv(i, logn), q);
    u32 t = N;
    for (u32 m = 1; m < N; m <<= 1) {
        t >>= 1;
        for (u32 i = 0; i < m; i++) {
            u32 j1 = 2 * i * t;
            u64 S = tw[m + i];
            for (u32 j = j1; j < j1 + t; j++) {
                u64 U = a[j], V = mulmod(a[j + t], S, q);
                a[j] = addmod(U, V, q);
                a[j + t] = submod(U, V, q);
            }
        }
    }
    free(tw);
}
/* Gentleman-Sande inverse, bit-reversed input, natural output, times N^-1
 * (Longa-Naehrig 2016, Alg. 2). */
static void intt_fast(u64 *a, u32 N, u64 q, u64 psi)
{
    u32 logn = ilog2(N);
    u64 pinv = invmod(psi, q);
    u64 *tw = (u64 *)malloc(sizeof(u64) * N); /* tw[i] = psi^-brv(i) */
    for (u32 i = 0; i < N; i++) tw[i] = powmod(pinv, brv(i, logn), q);
    u32 t = 1;
    for (u32 m = N; m > 1; m >>= 1) {
        u32 h = m >> 1, j1 = 0;
        for (u32 i = 0; i < h; i++) {
            u64 S = tw[h + i];
            for (u32 j = j1; j < j1 + t; j++) {
                u64 U = a[j], V = a[j + t];
                a[j] = addmod(U, V, q);
                a[j + t] = mulmod(submod(U, V, q), S, q);
            }
            j1 += 2 * t;
        }
        t <<= 1;
    }
    u64 ninv = invmod(N, q);
    for (u32 j = 0; j < N; j++) a[j] = mulmod(a[j], ninv, q);
    free(tw);
}
void oracle_ntt(const u64 *a, u32 N, u64 q, u64 psi, u64 *out)
{
    if (out != a) memcpy(out, a, sizeof(u64) * N);
    ntt_fast(out, N, q, psi);
}
void oracle_intt(const u64 *a, u32 N, u64 q, u64 psi, u64 *out)
{
    if (out != a) memcpy(out, a, sizeof(u64) * N);
    intt_fast(out, N, q, psi);
}

/* Schoolbook product in Z_q[X]/(X^N+1). */
void oracle_negacyclic_mul(const u64 *a, const u64 *b, u32 N, u64 q, u64 *out)
{
    memset(out, 0, sizeof(u64) * N);
    for (u32 i = 0; i < N; i++)
        for (u32 j = 0; j < N; j++) {
            u64 p = mulmod(a[i], b[j], q);
            if (i + j < N) out[i + j] = addmod(out[i + j], p, q);
            else out[i + j - N] = submod(out[i + j - N], p, q);
        }
}

/* Automorphism a(X) -> a(X^g) on coefficients, g odd: X^i -> (-1)^s X^(ig mod N)
 * where s = floor(ig / N) mod 2. */
void oracle_automorph_coeff(const u64 *a, u32 N, u64 q, u64 g, u64 *out)
{
    u64 twoN = 2ull * N;
    for (u32 i = 0; i < N; i++) {
        u64 e = ((u64)i * (g % twoN)) % twoN;
        if (e < N) out[e] = a[i] % q;
        else out[e - N] = submod(0, a[i] % q, q);
    }
}

/* Fast base conversion (Cheon et al. SAC 2018): for each target t,
 * out_t = sum_i [x_i * (Dhat_i)^-1]_{d_i} * (Dhat_i mod t) mod t,
 * Dhat_i = prod_{k != i} d_k.  in: [nfrom][N], out: [nto][N]. */
void oracle_bconv(const u64 *in, const u64 *from, u32 nfrom, const u64 *to, u32 nto, u32 N, u64 *out)
{
    for (u32 i = 0; i < nfrom; i++) {
        u64 dhat_mod_di = 1;
        for (u32 k = 0; k < nfrom; k++)
            if (k != i) dhat_mod_di = mulmod(dhat_mod_di, from[k] % from[i], from[i]);
        u64 inv = invmod(dhat_mod_di, from[i]);
        for (u32 t = 0; t < nto; t++) {
            u64 dhat_mod_t = 1;
            for (u32 k = 0; k < nfrom; k++)
                if (k != i) dhat_mod_t = mulmod(dhat_mod_t, from[k] % to[t], to[t]);
            for (u32 n = 0; n < N; n++) {
                u64 y = mulmod(in[(size_t)i * N + n], inv, from[i]);
                u64 prev = (i == 0) ? 0 : out[(size_t)t * N + n];
                out[(size_t)t * N + n] = addmod(prev, mulmod(y % to[t], dhat_mod_t, to[t]), to[t]);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Scheme context.                                                     */
/* ------------------------------------------------------------------ */
typedef struct oracle_ctx {
    u32 N, L, K, dnum, alpha, beta;
    u64 seed;
    u64 *mod; /* L+K moduli: q_0..q_{L-1}, p_0..p_{K-1} */
    u64 *psi; /* smallest primitive 2N-th root per modulus */
} oracle_ctx;

/* random-stream domains (nonce word 0) */
enum { DOM_SK = 1, DOM_PK_A = 2, DOM_PK_E = 3, DOM_KSK_A = 4, DOM_KSK_E = 5,
       DOM_ENC_V = 6, DOM_ENC_E0 = 7, DOM_ENC_E1 = 8 };

oracle_ctx *oracle_ctx_new(u32 N, const u64 *q, u32 L, const u64 *p, u32 K, u32 dnum, u64 seed)
{
    oracle_ctx *c = (oracle_ctx *)calloc(1, sizeof *c);
    c->N = N; c->L = L; c->K = K; c->dnum = dnum; c->seed = seed;
    c->alpha = (L + dnum - 1) / dnum;
    c->beta = (L + c->alpha - 1) / c->alpha;
    c->mod = (u64 *)malloc(sizeof(u64) * (L + K));
    c->psi = (u64 *)malloc(sizeof(u64) * (L + K));
    for (u32 i = 0; i < L; i++) c->mod[i] = q[i];
    for (u32 k = 0; k < K; k++) c->mod[L + k] = p[k];
    for (u32 i = 0; i < L + K; i++) c->psi[i] = oracle_min_psi(c->mod[i], N);
    return c;
}
void oracle_ctx_free(oracle_ctx *c)
{
    if (!c) return;
    free(c->mod); free(c->psi); free(c);
}
u32 oracle_ctx_alpha(const oracle_ctx *c) { return c->alpha; }
u32 oracle_ctx_beta(const oracle_ctx *c) { return c->beta; }
u64 oracle_ctx_psi(const oracle_ctx *c, u32 i) { return c->psi[i]; }

/* modulus index of limb i of a polynomial over Q_level followed by P */
static u32 qp_index(const oracle_ctx *c, u32 level, u32 i) { return i < level ? i : c->L + (i - level); }

/* signed integer polynomial -> residues over the listed modulus indices, then NTT */
static void int_to_eval(const oracle_ctx *c, const i64 *v, const u32 *midx, u32 n, u64 *out)
{
    for (u32 l = 0; l < n; l++) {
        u64 m = c->mod[midx[l]];
        u64 *o = out + (size_t)l * c->N;
        for (u32 k = 0; k < c->N; k++) o[k] = from_signed(v[k], m);
        ntt_fast(o, c->N, m, c->psi[midx[l]]);
    }
}

/* secret key: ternary coefficients from (seed, DOM_SK, 0); evaluation form over all L+K moduli */
void oracle_keygen_sk(const oracle_ctx *c, i64 *s_coeff, u64 *s_eval)
{
    u32 n = c->L + c->K;
    u32 *midx = (u32 *)malloc(sizeof(u32) * n);
    for (u32 i = 0; i < n; i++) midx[i] = i;
    oracle_sample_ternary(c->seed, DOM_SK, 0, c->N, s_coeff);
    int_to_eval(c, s_coeff, midx, n, s_eval);
    free(midx);
}

/* public key over Q_L: a uniform (drawn directly in the evaluation domain,
 * stream (seed, DOM_PK_A, limb)), e Gaussian (seed, DOM_PK_E, 0);
 * pk = (b, a) with b = -a*s + e.  pk: [2][L][N]. */
void oracle_keygen_pk(const oracle_ctx *c, const u64 *s_eval, u64 *pk)
{
    u32 N = c->N, L = c->L;
    i64 *e = (i64 *)malloc(sizeof(i64) * N);
    u32 *midx = (u32 *)malloc(sizeof(u32) * L);
    u64 *ee = (u64 *)malloc(sizeof(u64) * (size_t)L * N);
    for (u32 i = 0; i < L; i++) midx[i] = i;
    oracle_sample_gauss(c->seed, DOM_PK_E, 0, N, e);
    int_to_eval(c, e, midx, L, ee);
    for (u32 i = 0; i < L; i++) {
        u64 q = c->mod[i];
        u64 *a = pk + ((size_t)L + i) * N, *b = pk + (size_t)i * N;
        oracle_sample_uniform(c->seed, DOM_PK_A, i, N, q, a);
        for (u32 k = 0; k < N; k++)
            b[k] = addmod(submod(0, mulmod(a[k], s_eval[(size_t)i * N + k], q), q), ee[(size_t)i * N + k], q);
    }
    free(e); free(midx); free(ee);
}

/* Key-switching key from s_from to s, tagged `tag` (a Galois element, or 0
 * for relinearisation).  For each digit j < beta (limbs [j*alpha, (j+1)*alpha)
 * of Q_L) and each modulus m_i of Q_L u P:
 *   a_j[i]  uniform, stream (seed, DOM_KSK_A, tag<<32 | j<<16 | i), eval domain
 *   e_j     Gaussian, stream (seed, DOM_KSK_E, tag<<32 | j)
 *   b_j[i]  = -a_j[i]*s[i] + e_j[i] + [i in digit j] * (P mod q_i) * s_from[i]
 * i.e. b_j = -a_j s + e_j + P * Qhat_j * [Qhat_j^-1]_{Q_j} * s_from mod PQ.
 * ksk: [beta][2][L+K][N], component 0 = b, 1 = a. */
void oracle_keygen_ksk(const oracle_ctx *c, const u64 *s_eval, const u64 *sfrom_eval, u64 tag, u64 *ksk)
{
    u32 N = c->N, L = c->L, n = c->L + c->K;
    i64 *e = (i64 *)malloc(sizeof(i64) * N);
    u32 *midx = (u32 *)malloc(sizeof(u32) * n);
    u64 *ee = (u64 *)malloc(sizeof(u64) * (size_t)n * N);
    for (u32 i = 0; i < n; i++) midx[i] = i;
    for (u32 j = 0; j < c->beta; j++) {
        oracle_sample_gauss(c->seed, DOM_KSK_E, (tag << 32) | ((u64)j << 16), N, e);
        int_to_eval(c, e, midx, n, ee);
        u64 *B = ksk + ((size_t)j * 2 + 0) * n * N;
        u64 *A = ksk + ((size_t)j * 2 + 1) * n * N;
        for (u32 i = 0; i < n; i++) {
            u64 m = c->mod[i];
            u64 Pm = 1;
            for (u32 k = 0; k < c->K; k++) Pm = mulmod(Pm, c->mod[L + k] % m, m);
            int in_digit = (i < L) && (i / c->alpha == j);
            oracle_sample_uniform(c->seed, DOM_KSK_A, (tag << 32) | ((u64)j << 16) | i, N, m, A + (size_t)i * N);
            for (u32 k = 0; k < N; k++) {
                size_t o = (size_t)i * N + k;
                u64 v = addmod(submod(0, mulmod(A[o], s_eval[o], m), m), ee[o], m);
                if (in_digit) v = addmod(v, mulmod(Pm, sfrom_eval[o], m), m);
                B[o] = v;
            }
        }
    }
    free(e); free(midx); free(ee);
}

/* limb-wise conversions between evaluation and coefficient form; the limb
 * list is Q_level followed by `withP` ? P : nothing. */
static void to_coeff(const oracle_ctx *c, const u64 *in, u32 level, int withP, u64 *out)
{
    u32 n = level + (withP ? c->K : 0);
    for (u32 l = 0; l < n; l++) {
        u32 mi = qp_index(c, level, l);
        oracle_intt(in + (size_t)l * c->N, c->N, c->mod[mi], c->psi[mi], out + (size_t)l * c->N);
    }
}
static void to_eval(const oracle_ctx *c, const u64 *in, u32 level, int withP, u64 *out)
{
    u32 n = level + (withP ? c->K : 0);
    for (u32 l = 0; l < n; l++) {
        u32 mi = qp_index(c, level, l);
        oracle_ntt(in + (size_t)l * c->N, c->N, c->mod[mi], c->psi[mi], out + (size_t)l * c->N);
    }
}
void oracle_to_coeff(const oracle_ctx *c, const u64 *in, u32 level, int withP, u64 *out) { to_coeff(c, in, level, withP, out); }
void oracle_to_eval(const oracle_ctx *c, const u64 *in, u32 level, int withP, u64 *out) { to_eval(c, in, level, withP, out); }

/* sigma_g on an evaluation-form polynomial over Q_level (+P), by definition:
 * back to coefficients, X^i -> X^(ig), forward again. */
void oracle_automorph_eval(const oracle_ctx *c, const u64 *in, u32 level, int withP, u64 g, u64 *out)
{
    u32 N = c->N, n = level + (withP ? c->K : 0);
    u64 *t = (u64 *)malloc(sizeof(u64) * N), *t2 = (u64 *)malloc(sizeof(u64) * N);
    for (u32 l = 0; l < n; l++) {
        u32 mi = qp_index(c, level, l);
        oracle_intt(in + (size_t)l * N, N, c->mod[mi], c->psi[mi], t);
        oracle_automorph_coeff(t, N, c->mod[mi], g, t2);
        oracle_ntt(t2, N, c->mod[mi], c->psi[mi], out + (size_t)l * N);
    }
    free(t); free(t2);
}

/* sigma_g(s) over all L+K moduli (the source key of a rotation key) */
void oracle_galois_sk(const oracle_ctx *c, const u64 *s_eval, u64 g, u64 *out)
{
    oracle_automorph_eval(c, s_eval, c->L, 1, g, out);
}

/* ModUp of digit j at `level` (coefficient form in and out): digit limbs
 * D = [j*alpha, min((j+1)*alpha, level)) are copied, every other limb of
 * Q_level u P is the fast base conversion from D.  out: [level+K][N]. */
void oracle_modup(const oracle_ctx *c, const u64 *x_coeff, u32 level, u32 j, u64 *out)
{
    u32 N = c->N, K = c->K;
    u32 d0 = j * c->alpha, d1 = (j + 1) * c->alpha < level ? (j + 1) * c->alpha : level;
    u32 nd = d1 - d0, nt = level + K - nd;
    u64 *from = (u64 *)malloc(sizeof(u64) * nd), *to = (u64 *)malloc(sizeof(u64) * nt);
    u32 *tl = (u32 *)malloc(sizeof(u32) * nt);
    u64 *conv = (u64 *)malloc(sizeof(u64) * (size_t)nt * N);
    for (u32 i = 0; i < nd; i++) from[i] = c->mod[d0 + i];
    u32 t = 0;
    for (u32 l = 0; l < level + K; l++) {
        if (l >= d0 && l < d1) continue;
        tl[t] = l;
        to[t++] = c->mod[qp_index(c, level, l)];
    }
    oracle_bconv(x_coeff + (size_t)d0 * N, from, nd, to, nt, N, conv);
    for (u32 l = d0; l < d1; l++) memcpy(out + (size_t)l * N, x_coeff + (size_t)l * N, sizeof(u64) * N);
    for (u32 u = 0; u < nt; u++) memcpy(out + (size_t)tl[u] * N, conv + (size_t)u * N, sizeof(u64) * N);
    free(from); free(to); free(tl); free(conv);
}

/* ModDown (coefficient form): x over Q_level u P -> (x_i - BConv_{P->q_i}(x_P)) * P^-1 mod q_i. */
void oracle_moddown(const oracle_ctx *c, const u64 *x_coeff, u32 level, u64 *out)
{
    u32 N = c->N, K = c->K;
    u64 *conv = (u64 *)malloc(sizeof(u64) * (size_t)level * N);
    oracle_bconv(x_coeff + (size_t)level * N, c->mod + c->L, K, c->mod, level, N, conv);
    for (u32 i = 0; i < level; i++) {
        u64 q = c->mod[i], Pm = 1;
        for (u32 k = 0; k < K; k++) Pm = mulmod(Pm, c->mod[c->L + k] % q, q);
        u64 Pinv = invmod(Pm, q);
        for (u32 n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            out[o] = mulmod(submod(x_coeff[o], conv[o], q), Pinv, q);
        }
    }
    free(conv);
}

/* Hybrid key switching of one evaluation-form polynomial d over Q_level:
 *   1. to coefficients;  2. per digit j < ceil(level/alpha): ModUp, then NTT
 *   over Q_level u P;  3. acc_b = sum_j dhat_j * ksk[j][b] (limbs of Q_level
 *   and P);  4. ModDown of acc_0, acc_1.
 * out: [2][level][N] evaluation form. */
void oracle_keyswitch(const oracle_ctx *c, const u64 *d_eval, u32 level, const u64 *ksk, u64 *out)
{
    u32 N = c->N, K = c->K, n = level + K, nall = c->L + c->K;
    u32 beta = (level + c->alpha - 1) / c->alpha;
    u64 *dc = (u64 *)malloc(sizeof(u64) * (size_t)level * N);
    u64 *up = (u64 *)malloc(sizeof(u64) * (size_t)n * N);
    u64 *upe = (u64 *)malloc(sizeof(u64) * (size_t)n * N);
    u64 *acc = (u64 *)calloc((size_t)2 * n * N, sizeof(u64));
    u64 *accc = (u64 *)malloc(sizeof(u64) * (size_t)n * N);
    u64 *md = (u64 *)malloc(sizeof(u64) * (size_t)level * N);
    to_coeff(c, d_eval, level, 0, dc);
    for (u32 j = 0; j < beta; j++) {
        oracle_modup(c, dc, level, j, up);
        to_eval(c, up, level, 1, upe);
        for (u32 b = 0; b < 2; b++)
            for (u32 l = 0; l < n; l++) {
                u32 mi = qp_index(c, level, l);
                u64 m = c->mod[mi];
                const u64 *kk = ksk + (((size_t)j * 2 + b) * nall + mi) * N;
                u64 *a = acc + ((size_t)b * n + l) * N;
                for (u32 k = 0; k < N; k++) a[k] = addmod(a[k], mulmod(upe[(size_t)l * N + k], kk[k], m), m);
            }
    }
    for (u32 b = 0; b < 2; b++) {
        to_coeff(c, acc + (size_t)b * n * N, level, 1, accc);
        oracle_moddown(c, accc, level, md);
        to_eval(c, md, level, 0, out + (size_t)b * level * N);
    }
    free(dc); free(up); free(upe); free(acc); free(accc); free(md);
}

/* Rotation by Galois element g: (c0, c1) -> (sigma(c0), sigma(c1)), then
 * key switching of sigma(c1) from sigma_g(s) back to s:
 * out = (sigma(c0) + ks_0, ks_1). */
void oracle_rotate(const oracle_ctx *c, const u64 *ct, u32 level, u64 g, const u64 *ksk, u64 *out)
{
    size_t pl = (size_t)level * c->N;
    u64 *sc = (u64 *)malloc(sizeof(u64) * 2 * pl);
    u64 *ks = (u64 *)malloc(sizeof(u64) * 2 * pl);
    oracle_automorph_eval(c, ct, level, 0, g, sc);
    oracle_automorph_eval(c, ct + pl, level, 0, g, sc + pl);
    oracle_keyswitch(c, sc + pl, level, ksk, ks);
    for (u32 i = 0; i < level; i++)
        for (u32 k = 0; k < c->N; k++) {
            size_t o = (size_t)i * c->N + k;
            out[o] = addmod(sc[o], ks[o], c->mod[i]);
            out[pl + o] = ks[pl + o];
        }
    free(sc); free(ks);
}

/* Hoisted rotations of one ciphertext (Halevi-Shoup hoisting, in the hybrid
 * key-switching form): the digits of c1 are raised once -- coefficients, ModUp
 * of every digit, NTT over Q_level u P -- and rotation r applies sigma_{g_r}
 * to the raised digits in the evaluation domain, then takes the key inner
 * product and ModDown of oracle_keyswitch: out_r = (sigma(c0) + ks_0, ks_1).
 * sigma_g(ModUp(x)) lifts sigma_g(x) with the same digit bound, but the fast
 * base conversion is not odd (BConv(-x) != -BConv(x)), so for g != 1 the
 * residues differ from those of oracle_rotate.
 * gs: [n]; ksks: [n][beta_max][2][L+K][N]; out: [n][2][level][N]. */
void oracle_rotate_hoisted(const oracle_ctx *c, const u64 *ct, u32 level, const u64 *gs, u32 n, const u64 *ksks,
                           u64 *out)
{
    u32 N = c->N, K = c->K, nl = level + K, nall = c->L + c->K;
    u32 beta = (level + c->alpha - 1) / c->alpha;
    size_t pl = (size_t)level * N, limbs = (size_t)nl * N, keysz = (size_t)c->beta * 2 * nall * N;
    u64 *dc = (u64 *)malloc(sizeof(u64) * pl);
    u64 *up = (u64 *)malloc(sizeof(u64) * limbs);
    u64 *ext = (u64 *)malloc(sizeof(u64) * beta * limbs);
    u64 *d = (u64 *)malloc(sizeof(u64) * limbs);
    u64 *acc = (u64 *)malloc(sizeof(u64) * 2 * limbs);
    u64 *accc = (u64 *)malloc(sizeof(u64) * limbs);
    u64 *md = (u64 *)malloc(sizeof(u64) * pl);
    u64 *ks = (u64 *)malloc(sizeof(u64) * 2 * pl);
    u64 *sc0 = (u64 *)malloc(sizeof(u64) * pl);
    /* the raised digits, once */
    to_coeff(c, ct + pl, level, 0, dc);
    for (u32 j = 0; j < beta; j++) {
        oracle_modup(c, dc, level, j, up);
        to_eval(c, up, level, 1, ext + j * limbs);
    }
    for (u32 r = 0; r < n; r++) {
        const u64 *ksk = ksks + r * keysz;
        memset(acc, 0, sizeof(u64) * 2 * limbs);
        for (u32 j = 0; j < beta; j++) {
            oracle_automorph_eval(c, ext + j * limbs, level, 1, gs[r], d);
            for (u32 b = 0; b < 2; b++)
                for (u32 l = 0; l < nl; l++) {
                    u32 mi = qp_index(c, level, l);
                    u64 m = c->mod[mi];
                    const u64 *kk = ksk + (((size_t)j * 2 + b) * nall + mi) * N;
                    u64 *a = acc + ((size_t)b * nl + l) * N;
                    for (u32 k = 0; k < N; k++) a[k] = addmod(a[k], mulmod(d[(size_t)l * N + k], kk[k], m), m);
                }
        }
        for (u32 b = 0; b < 2; b++) {
            to_coeff(c, acc + (size_t)b * limbs, level, 1, accc);
            oracle_moddown(c, accc, level, md);
            to_eval(c, md, level, 0, ks + (size_t)b * pl);
        }
        oracle_automorph_eval(c, ct, level, 0, gs[r], sc0);
        u64 *o = out + (size_t)r * 2 * pl;
        for (u32 i = 0; i < level; i++)
            for (u32 k = 0; k < N; k++) {
                size_t x = (size_t)i * N + k;
                o[x] = addmod(sc0[x], ks[x], c->mod[i]);
                o[pl + x] = ks[pl + x];
            }
    }
    free(dc); free(up); free(ext); free(d); free(acc); free(accc); free(md); free(ks); free(sc0);
}

/* Ciphertext product (the multiplications of paper Alg. 4's Chebyshev
 * evaluation, OpenFHE's EvalMult): the tensor (d0, d1, d2) = (a0 b0,
 * a0 b1 + a1 b0, a1 b1) decrypts under (1, s, s^2); d2 is key-switched from
 * s^2 to s with the relinearisation key (oracle_keygen_ksk with s_from = s^2,
 * tag 0): out = (d0 + ks_0, d1 + ks_1).  No rescale.  out: [2][level][N]. */
void oracle_mul_relin(const oracle_ctx *c, const u64 *a, const u64 *b, u32 level, const u64 *rlk, u64 *out)
{
    size_t pl = (size_t)level * c->N;
    u64 *d = (u64 *)malloc(sizeof(u64) * 3 * pl);
    u64 *ks = (u64 *)malloc(sizeof(u64) * 2 * pl);
    for (u32 i = 0; i < level; i++) {
        u64 q = c->mod[i];
        for (u32 k = 0; k < c->N; k++) {
            size_t o = (size_t)i * c->N + k;
            d[o] = mulmod(a[o], b[o], q);
            d[pl + o] = addmod(mulmod(a[o], b[pl + o], q), mulmod(a[pl + o], b[o], q), q);
            d[2 * pl + o] = mulmod(a[pl + o], b[pl + o], q);
        }
    }
    oracle_keyswitch(c, d + 2 * pl, level, rlk, ks);
    for (u32 i = 0; i < level; i++)
        for (u32 k = 0; k < c->N; k++) {
            size_t o = (size_t)i * c->N + k;
            out[o] = addmod(d[o], ks[o], c->mod[i]);
            out[pl + o] = addmod(d[pl + o], ks[pl + o], c->mod[i]);
        }
    free(d); free(ks);
}

/* out = v * ct for an integer v: every residue times (v mod q_i). */
void oracle_mul_int(const oracle_ctx *c, const u64 *ct, u32 level, i64 v, u64 *out)
{
    size_t pl = (size_t)level * c->N;
    for (u32 b = 0; b < 2; b++)
        for (u32 i = 0; i < level; i++) {
            u64 q = c->mod[i], vm = from_signed(v, q);
            for (u32 k = 0; k < c->N; k++) {
                size_t o = b * pl + (size_t)i * c->N + k;
                out[o] = mulmod(ct[o], vm, q);
            }
        }
}

/* c0 += v: the constant polynomial v takes the value v at every evaluation
 * point, so every residue of c0 limb i gains (v mod q_i); c1 is copied. */
void oracle_add_int(const oracle_ctx *c, const u64 *ct, u32 level, i64 v, u64 *out)
{
    size_t pl = (size_t)level * c->N;
    for (u32 i = 0; i < level; i++) {
        u64 q = c->mod[i], vm = from_signed(v, q);
        for (u32 k = 0; k < c->N; k++) {
            size_t o = (size_t)i * c->N + k;
            out[o] = addmod(ct[o], vm, q);
            out[pl + o] = ct[pl + o];
        }
    }
}

/* Chebyshev interpolant of f(z) = beta * max(0, z) on [-1, 1] (paper Sec. 5.6
 * and Alg. 4: the input is scaled by 1/beta first, f is evaluated by a
 * degree-D Chebyshev series), at the D+1 Chebyshev nodes
 * z_k = cos(theta_k), theta_k = pi (k + 1/2) / (D + 1):
 *   c_d = (2 / (D + 1)) sum_k f(z_k) cos(d theta_k), and c_0 halved,
 * the sums taken in order k = 0..D in binary64.  out: [D + 1]. */
void oracle_cheb_coeffs(double beta, u32 D, double *out)
{
    for (u32 d = 0; d <= D; d++) {
        double sum = 0.0;
        for (u32 k = 0; k <= D; k++) {
            double th = M_PI * ((double)k + 0.5) / (double)(D + 1);
            double z = cos(th);
            double f = z < 0.0 ? 0.0 : beta * z;
            sum += f * cos((double)d * th);
        }
        out[d] = sum * 2.0 / (double)(D + 1);
    }
    out[0] *= 0.5;
}

/* Chebyshev interpolant of the scaled cosine of bootstrapping's modular
 * reduction, f(z) = cos(2 pi (K z - 1/4) / 2^r) on [-1, 1] (so that r
 * double-angle steps give sin(2 pi K z)), at the same D+1 nodes and with the
 * same coefficient formula as oracle_cheb_coeffs. */
void oracle_cos_cheb_coeffs(double K, u32 r, u32 D, double *out)
{
    for (u32 d = 0; d <= D; d++) {
        double sum = 0.0;
        for (u32 k = 0; k <= D; k++) {
            double th = M_PI * ((double)k + 0.5) / (double)(D + 1);
            double z = cos(th);
            double f = cos((2.0 * M_PI) * (K * z - 0.25) / ldexp(1.0, (int)r));
            sum += f * cos((double)d * th);
        }
        out[d] = sum * 2.0 / (double)(D + 1);
    }
    out[0] *= 0.5;
}

/* round half away from zero (the encoding of a constant c at scale D is
 * llround(c * D)) */
i64 oracle_llround(double x) { return llround(x); }

/* The integer K a constant c is encoded as before a rescale by q_{level-1}, so
 * that the rescaled product has scale `target`: a ciphertext of scale `scale`
 * times K, divided by q_{level-1}, has scale scale * K / q ~= c * target.
 * K = llround(((c * target) * q_{level-1}) / scale) in binary64. */
i64 oracle_const_factor(const oracle_ctx *c, u32 level, double cval, double target, double scale)
{
    return llround(((cval * target) * (double)c->mod[level - 1]) / scale);
}

/* pk encryption of an integer message polynomial m (coefficients), at level L:
 * v ternary (DOM_ENC_V), e0, e1 Gaussian (DOM_ENC_E0/E1), all with idx = nonce;
 * ct = (v*pk0 + e0 + m, v*pk1 + e1).  ct: [2][L][N]. */
void oracle_encrypt(const oracle_ctx *c, const u64 *pk, const i64 *m, u64 nonce, u64 *ct)
{
    u32 N = c->N, L = c->L;
    i64 *v = (i64 *)malloc(sizeof(i64) * N), *e0 = (i64 *)malloc(sizeof(i64) * N), *e1 = (i64 *)malloc(sizeof(i64) * N);
    u32 *midx = (u32 *)malloc(sizeof(u32) * L);
    u64 *V = (u64 *)malloc(sizeof(u64) * (size_t)L * N), *E0 = (u64 *)malloc(sizeof(u64) * (size_t)L * N);
    u64 *E1 = (u64 *)malloc(sizeof(u64) * (size_t)L * N), *M = (u64 *)malloc(sizeof(u64) * (size_t)L * N);
    for (u32 i = 0; i < L; i++) midx[i] = i;
    oracle_sample_ternary(c->seed, DOM_ENC_V, nonce, N, v);
    oracle_sample_gauss(c->seed, DOM_ENC_E0, nonce, N, e0);
    oracle_sample_gauss(c->seed, DOM_ENC_E1, nonce, N, e1);
    int_to_eval(c, v, midx, L, V);
    int_to_eval(c, e0, midx, L, E0);
    int_to_eval(c, e1, midx, L, E1);
    int_to_eval(c, m, midx, L, M);
    size_t pl = (size_t)L * N;
    for (u32 i = 0; i < L; i++)
        for (u32 k = 0; k < N; k++) {
            size_t o = (size_t)i * N + k;
            u64 q = c->mod[i];
            ct[o] = addmod(addmod(mulmod(V[o], pk[o], q), E0[o], q), M[o], q);
            ct[pl + o] = addmod(mulmod(V[o], pk[pl + o], q), E1[o], q);
        }
    free(v); free(e0); free(e1); free(midx); free(V); free(E0); free(E1); free(M);
}

/* integer polynomial -> evaluation-form plaintext over Q_level */
void oracle_plain_from_coeffs(const oracle_ctx *c, const i64 *m, u32 level, u64 *pt)
{
    u32 *midx = (u32 *)malloc(sizeof(u32) * level);
    for (u32 i = 0; i < level; i++) midx[i] = i;
    int_to_eval(c, m, midx, level, pt);
    free(midx);
}

/* m = c0 + c1*s over Q_level, evaluation form */
void oracle_decrypt(const oracle_ctx *c, const u64 *s_eval, const u64 *ct, u32 level, u64 *m)
{
    size_t pl = (size_t)level * c->N;
    for (u32 i = 0; i < level; i++)
        for (u32 k = 0; k < c->N; k++) {
            size_t o = (size_t)i * c->N + k;
            m[o] = addmod(ct[o], mulmod(ct[pl + o], s_eval[o], c->mod[i]), c->mod[i]);
        }
}

void oracle_mul_plain(const oracle_ctx *c, const u64 *ct, const u64 *pt, u32 level, u64 *out)
{
    size_t pl = (size_t)level * c->N;
    for (u32 b = 0; b < 2; b++)
        for (u32 i = 0; i < level; i++)
            for (u32 k = 0; k < c->N; k++) {
                size_t o = (size_t)i * c->N + k;
                out[b * pl + o] = mulmod(ct[b * pl + o], pt[o], c->mod[i]);
            }
}
void oracle_add(const oracle_ctx *c, const u64 *x, const u64 *y, u32 level, u64 *out)
{
    size_t pl = (size_t)level * c->N;
    for (u32 b = 0; b < 2; b++)
        for (u32 i = 0; i < level; i++)
            for (u32 k = 0; k < c->N; k++) {
                size_t o = b * pl + (size_t)i * c->N + k;
                out[o] = addmod(x[o], y[o], c->mod[i]);
            }
}

/* Floor rescale of an evaluation-form polynomial over Q_level by the last prime
 * q_t = q_{level-1}: r = [x]_{q_t} in [0, q_t) (coefficients), then
 * out_i = (x_i - r) * q_t^-1 mod q_i for i < level-1, i.e. (x - r)/q_t. */
void oracle_rescale_poly(const oracle_ctx *c, const u64 *x, u32 level, u64 *out)
{
    u32 N = c->N, t = level - 1;
    u64 qt = c->mod[t];
    u64 *r = (u64 *)malloc(sizeof(u64) * N), *ri = (u64 *)malloc(sizeof(u64) * N);
    oracle_intt(x + (size_t)t * N, N, qt, c->psi[t], r);
    for (u32 i = 0; i < t; i++) {
        u64 q = c->mod[i], inv = invmod(qt % q, q);
        for (u32 k = 0; k < N; k++) ri[k] = r[k] % q;
        oracle_ntt(ri, N, q, c->psi[i], ri);
        for (u32 k = 0; k < N; k++) {
            size_t o = (size_t)i * N + k;
            out[o] = mulmod(submod(x[o], ri[k], q), inv, q);
        }
    }
    free(r); free(ri);
}
void oracle_rescale(const oracle_ctx *c, const u64 *ct, u32 level, u64 *out)
{
    size_t pin = (size_t)level * c->N, pout = (size_t)(level - 1) * c->N;
    oracle_rescale_poly(c, ct, level, out);
    oracle_rescale_poly(c, ct + pin, level, out + pout);
}

/* ------------------------------------------------------------------ */
/* Canonical embedding (paper Sec. 3.2: C^{N/2} <-> R).                */
/* slot i <-> evaluation at zeta^(5^i mod 2N), zeta = exp(i*pi/N).     */
/* ------------------------------------------------------------------ */

/* m_k = round(scale * (2/N) * Re(sum_i z_i * zeta^(-5^i k))), k < N; round
 * half away from zero.  nslots <= N/2 (missing slots are zero).  Returns 0,
 * or -1 when a coefficient does not fit in 63 bits.  O(N * nslots). */
int oracle_encode(u32 N, const double *zr, const double *zi, u32 nslots, double scale, i64 *m)
{
    u64 twoN = 2ull * N;
    double *cs = (double *)malloc(sizeof(double) * twoN), *sn = (double *)malloc(sizeof(double) * twoN);
    u64 *g = (u64 *)malloc(sizeof(u64) * (nslots ? nslots : 1));
    for (u64 e = 0; e < twoN; e++) { cs[e] = cos(M_PI * (double)e / (double)N); sn[e] = sin(M_PI * (double)e / (double)N); }
    u64 p = 1;
    for (u32 i = 0; i < nslots; i++) { g[i] = p; p = (p * 5) % twoN; }
    int rc = 0;
    for (u32 k = 0; k < N; k++) {
        double acc = 0.0;
        for (u32 i = 0; i < nslots; i++) {
            u64 e = (twoN - (g[i] * k) % twoN) % twoN; /* zeta^(-5^i k) */
            acc += zr[i] * cs[e] - zi[i] * sn[e];
        }
        double v = scale * (2.0 / (double)N) * acc;
        double r = round(v);
        if (!(fabs(r) < 9.2e18)) { rc = -1; r = 0; }
        m[k] = (i64)r;
    }
    free(cs); free(sn); free(g);
    return rc;
}

/* z_i = (1/scale) * sum_k m_k * zeta^(5^i k), for i < nslots; m as doubles. */
void oracle_decode(u32 N, const double *m, u32 nslots, double scale, double *zr, double *zi)
{
    u64 twoN = 2ull * N;
    double *cs = (double *)malloc(sizeof(double) * twoN), *sn = (double *)malloc(sizeof(double) * twoN);
    for (u64 e = 0; e < twoN; e++) { cs[e] = cos(M_PI * (double)e / (double)N); sn[e] = sin(M_PI * (double)e / (double)N); }
    u64 g = 1;
    for (u32 i = 0; i < nslots; i++) {
        double ar = 0.0, ai = 0.0;
        for (u32 k = 0; k < N; k++) {
            u64 e = (g * k) % twoN;
            ar += m[k] * cs[e];
            ai += m[k] * sn[e];
        }
        zr[i] = ar / scale;
        zi[i] = ai / scale;
        g = (g * 5) % twoN;
    }
    free(cs); free(sn);
}

/* c0 += pt over Q_level (plaintext addition; c1 unchanged) */
void oracle_add_plain(const oracle_ctx *c, const u64 *ct, const u64 *pt, u32 level, u64 *out)
{
    size_t pl = (size_t)level * c->N;
    for (u32 i = 0; i < level; i++)
        for (u32 k = 0; k < c->N; k++) {
            size_t o = (size_t)i * c->N + k;
            out[o] = addmod(ct[o], pt[o], c->mod[i]);
            out[pl + o] = ct[pl + o];
        }
}
