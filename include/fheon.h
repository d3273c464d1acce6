/*
 * fheon.h -- C ABI of the GB300 (sm_103a) RNS-CKKS rotation library behind
 * FHEON's encrypted CNN layers (arxiv 2510.03996).
 *
 * FHEON (paper Sec. 5.7, "Support Functions") exposes context generation,
 * key generation and key management, an encryption layer, the secure CNN
 * layers of Sec. 5 and bootstrapping on top of RNS-CKKS (Sec. 3.2).  This
 * library is the GPU arithmetic under those calls: the homomorphic rotation
 * (Galois automorphism + hybrid key switching) and the plaintext-multiply,
 * add and rescale steps around it, and on top of them the secure layers as
 * prepared handles (the special convolution of Sec. 5.3; packed convolution,
 * pooling and FC of Sec. 5.1-5.5; the Chebyshev ReLU of Sec. 5.6; repacking),
 * CKKS bootstrapping as a layer, model programs and a continuous-batching
 * server.
 *
 * Conventions shared by every call
 *  - Every call returns int: FHEON_OK (0) or a negative FHEON_ERR_* code;
 *    fheon_last_error() gives a message for the last failing call on a
 *    context.  No call aborts the process.
 *  - Results are returned through out-parameters.  Every handle (context,
 *    keys, plaintext, ciphertext, layer) is owned by the caller and freed
 *    with its matching *_destroy; destroying NULL is a no-op.
 *  - Device memory comes from the allocator installed by
 *    fheon_set_allocator() (default: cudaMalloc/cudaFree).  All device
 *    work of a context is enqueued on its stream (a cudaStream_t passed as
 *    void*; NULL = the legacy default stream) and is asynchronous, except
 *    the calls documented as blocking (downloads, decode, fheon_sync).
 *  - Polynomials live on the device limb-major: u64[limbs][N], residues in
 *    [0, m_i), in the evaluation (NTT) domain, slot j holding
 *    a(psi_i^(2*brv(j)+1)) for the smallest primitive 2N-th root psi_i of
 *    m_i.  A ciphertext at level l is u64[2][l][N] over q_0..q_{l-1}.
 *    Host arrays passed to upload/download use the same layout.
 *  - Slot i of a plaintext is the evaluation at zeta^(5^i mod 2N),
 *    zeta = exp(i*pi/N); rotating by r moves slot i+r to slot i (r > 0 is
 *    a left rotation), Galois element 5^r mod 2N.
 *  - Supported sizes: N = 2^10 .. 2^17; primes of at most 61 bits with
 *    q = 1 (mod 2N); digit count, digit size and P count each at most 16.
 */
#ifndef FHEON_H
#define FHEON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Errors                                                             */
/* ------------------------------------------------------------------ */
#define FHEON_OK 0
#define FHEON_ERR_ARG (-1)           /* bad argument, size or handle */
#define FHEON_ERR_OOM (-2)           /* the allocator returned NULL */
#define FHEON_ERR_NO_KEY (-3)        /* rotation key for that step missing */
#define FHEON_ERR_LEVEL (-4)         /* operand levels incompatible */
#define FHEON_ERR_SCALE (-5)         /* operand scales incompatible */
#define FHEON_ERR_TIMEOUT (-6)       /* a bounded device wait ran out */
#define FHEON_ERR_CUDA (-7)          /* a CUDA runtime call failed */
#define FHEON_ERR_UNIMPLEMENTED (-8) /* not available in this build */
#define FHEON_PENDING 1              /* not an error: the request is still running */

typedef struct fheon_ctx fheon_ctx;
typedef struct fheon_sk fheon_sk;
typedef struct fheon_pk fheon_pk;
typedef struct fheon_pt fheon_pt;
typedef struct fheon_ct fheon_ct;
typedef struct fheon_layer fheon_layer;
typedef struct fheon_model fheon_model;
typedef struct fheon_server fheon_server;
/* Packed layout of a feature map (C, H, W) in the slots: channel c in the
 * block at offset c * block; position (i, j) at c*block + dil*(i*grid + j).
 * `grid` is the row stride; `dil` the spacing of valid positions (a stride-s
 * layer multiplies it by s, leaving its outputs in place). */
typedef struct fheon_map {
    uint32_t C, H, W, grid, dil, block;
} fheon_map;

/* Message for an error code (static storage). */
const char *fheon_error_string(int code);
/* Message of the last failing call on ctx (valid until the next call).
 * A call that rejects its arguments outright (a null pointer, a size out of
 * range) returns FHEON_ERR_ARG and leaves the message as it was; every
 * other failure sets it. */
const char *fheon_last_error(const fheon_ctx *ctx);

/* ------------------------------------------------------------------ */
/* Device memory                                                      */
/* ------------------------------------------------------------------ */
/* Allocation hook: returns device memory of `bytes` usable on `stream`,
 * or NULL (the calling API function then fails with FHEON_ERR_OOM). */
typedef void *(*fheon_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*fheon_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
/* Install the process-wide allocator used for every later allocation
 * (NULL, NULL restores cudaMalloc/cudaFree).  Memory is freed through the
 * hook that allocated it, so a free_fn (and its `user`) must stay callable
 * until every block it allocated has been released. */
int fheon_set_allocator(fheon_alloc_fn alloc, fheon_free_fn free_fn, void *user);

/* ------------------------------------------------------------------ */
/* Context (paper Sec. 5.7, context generation)                         */
/* ------------------------------------------------------------------ */
/* Create a context for ring degree N with ciphertext moduli q[0..nq) and
 * special moduli p[0..np), hybrid key switching with `dnum` digits
 * (paper Sec. 6: "4 digits"; digit j = limbs [j*alpha, (j+1)*alpha) of Q,
 * alpha = ceil(nq/dnum)), default scale `scale` and master seed `seed`
 * (every random draw is ChaCha20 on (seed, purpose, index)).  Moduli must
 * be distinct primes = 1 mod 2N.  Uploads all constant tables on `stream`.
 * Errors: FHEON_ERR_ARG for unsupported sizes or non-NTT-friendly moduli. */
int fheon_ctx_create(uint32_t N, const uint64_t *q, uint32_t nq, const uint64_t *p, uint32_t np,
                     uint32_t dnum, double scale, uint64_t seed, void *stream, fheon_ctx **out);
/* As fheon_ctx_create, choosing the moduli from bit sizes: for each size in
 * the order qbits then pbits, the largest unused prime q < 2^bits with
 * q = 1 (mod 2N). */
int fheon_ctx_create_bits(uint32_t N, const uint32_t *qbits, uint32_t nq, const uint32_t *pbits,
                          uint32_t np, uint32_t dnum, double scale, uint64_t seed, void *stream,
                          fheon_ctx **out);
int fheon_ctx_destroy(fheon_ctx *ctx);
/* Host-only parameter calls (no device, no context).  The moduli
 * fheon_ctx_create_bits picks for these bit sizes, in order, into out[n]:
 * for each size, the largest unused prime below 2^bits that is 1 mod 2N.
 * FHEON_ERR_ARG for N outside the supported powers of two, a size outside
 * [20, 61], or a size with no such prime. */
int fheon_pick_primes(uint32_t N, const uint32_t *bits, uint32_t n, uint64_t *out);
/* The NTT's root for modulus q: the smallest primitive 2N-th root of unity
 * mod q (the minimum over the odd powers of any one).  0 when q is not a
 * prime = 1 mod 2N or N not a power of two. */
uint64_t fheon_min_root(uint64_t q, uint32_t N);
/* The discrete Gaussian sampler's table (sigma 3.2, tail 20): out[k + 20] =
 * floor(2^64 * sum_{i <= k} rho(i) / sum rho) for k < 20, rho(k) =
 * exp(-k^2 / (2 sigma^2)) in binary64, out[40] = 0; n must be 41. */
int fheon_gaussian_cdt(uint64_t *out, uint32_t n);
/* N, L (= nq), K (= np), alpha (limbs per digit), beta (digits at level L). */
int fheon_ctx_info(const fheon_ctx *ctx, uint32_t *N, uint32_t *L, uint32_t *K, uint32_t *alpha,
                   uint32_t *beta);
/* The L+K moduli, Q first, into out[L+K]. */
int fheon_ctx_moduli(const fheon_ctx *ctx, uint64_t *out);
int fheon_ctx_set_stream(fheon_ctx *ctx, void *stream);
/* Key-switching schedule (results are identical under every schedule; only
 * speed differs).  Bits: 1 = plain second NTT pass plus a streaming key
 * inner-product kernel (else the inner product is summed inside the second
 * pass); 2 = ModUp base conversion tiled per digit (needs alpha <= 4);
 * 4 = ModDown base conversion tiled per component (needs K <= 4); 8 = the
 * streaming inner product fed by TMA bulk copies into shared memory (needs
 * bit 1); 16 = the NTT's row passes at radix 8 on 2048-element tiles (half
 * the registers a thread, one more CTA per SM) instead of radix 16 on
 * 4096-element tiles (needs bit 1).  The default is 9.  get returns the
 * current value; set fails with FHEON_ERR_ARG for values outside
 * [0, FHEON_NUM_SCHEDULES) and bits the parameters do not allow. */
#define FHEON_NUM_SCHEDULES 32
int fheon_ctx_get_schedule(const fheon_ctx *ctx, int *schedule);
int fheon_ctx_set_schedule(fheon_ctx *ctx, int schedule);
/* Batching switch.  on = 1 (the default): batched rotations and products
 * (fheon_rotate_batch, the layers, series and bootstraps built on them) run
 * as one launch sequence over the whole batch, with the rotations of one
 * input hoisted.  on = 0: the plain one-ciphertext-per-launch path, every
 * rotation and product of a batch through its own launch sequence, none
 * hoisted (its results are the plain rotation's; a hoisted rotation differs
 * from it in the low bits).  For measuring what batching gains.
 * FHEON_ERR_ARG for other values. */
int fheon_ctx_set_batching(fheon_ctx *ctx, int on);
/* Autotuner: time every schedule the parameters allow on the caller's batch
 * (one untimed run, then `reps` timed runs of fheon_rotate_batch with CUDA
 * events on the context's stream), keep the fastest on the context and
 * return it in *best.  ms_per_batch, when not NULL, receives
 * FHEON_NUM_SCHEDULES entries indexed by schedule (negative for schedules not
 * allowed).  The batch's outputs are overwritten.  Blocking. */
int fheon_autotune_schedule(fheon_ctx *ctx, const struct fheon_rot_item *items, uint32_t n, uint32_t reps, int *best,
                            double *ms_per_batch);
/* Block until all work enqueued on the context's stream is done.  Returns
 * FHEON_ERR_TIMEOUT (once) when a kernel's bounded wait on its own copies ran
 * out since the last check; the outputs of that work are then not valid.  The
 * download calls check the same way. */
int fheon_sync(fheon_ctx *ctx);

/* ------------------------------------------------------------------ */
/* Keys (paper Sec. 5.7, key generation and evaluation-key management)  */
/* ------------------------------------------------------------------ */
/* Secret key s (ternary, stream (seed, 1, 0)) and public key
 * (b, a) = (-a*s + e, a) over Q_L; a uniform in the evaluation domain
 * (stream (seed, 2, limb)), e discrete Gaussian sigma = 3.2 tail 20
 * (stream (seed, 3, 0)).  Generated on the device. */
int fheon_keygen(fheon_ctx *ctx, fheon_sk **sk, fheon_pk **pk);
int fheon_sk_destroy(fheon_sk *sk);
int fheon_pk_destroy(fheon_pk *pk);
/* Blocking copy of s (evaluation form over all L+K moduli, u64[L+K][N]). */
int fheon_sk_download(fheon_ctx *ctx, const fheon_sk *sk, uint64_t *host);
/* Blocking copy of pk, u64[2][L][N] (b then a), canonical residues. */
int fheon_pk_download(fheon_ctx *ctx, const fheon_pk *pk, uint64_t *host);

/* Rotation keys for slot rotations steps[0..n) (Galois elements 5^r mod 2N;
 * paper Sec. 5.7: the rotation indices each layer needs).  A key for g is
 * beta digits of (b_j, a_j) over Q_L u P with
 *   b_j = -a_j*s + e_j + [limb in digit j] * P * sigma_g(s),
 * a_j uniform (stream (seed, 4, g<<32 | j<<16 | limb)), e_j Gaussian
 * (stream (seed, 5, g<<32 | j<<16)).  Keys stay resident on the device;
 * existing keys are kept. */
int fheon_rotkeygen(fheon_ctx *ctx, const fheon_sk *sk, const int32_t *steps, uint32_t n);
/* Relinearisation key: the key-switching key from s^2 to s (b_j = -a_j s +
 * e_j + P [limb in digit j] s^2, streams tagged 0), kept on the context; the
 * ciphertext product needs it.  A second call does nothing. */
int fheon_relinkeygen(fheon_ctx *ctx, const fheon_sk *sk);
/* Same, by Galois element (odd g < 2N; 2N-1 is complex conjugation). */
int fheon_galois_keygen(fheon_ctx *ctx, const fheon_sk *sk, const uint64_t *galois, uint32_t n);
/* Drop the key of Galois element g (paper Sec. 5.7: keys loaded and cleared
 * per block); FHEON_ERR_NO_KEY if absent.  Waits for the context's queued
 * work; a layer graph captured with this key must not be replayed after. */
int fheon_key_erase(fheon_ctx *ctx, uint64_t galois);
/* Number of resident rotation keys and their device bytes. */
int fheon_key_stats(const fheon_ctx *ctx, uint32_t *count, uint64_t *bytes);
/* Blocking copy of the key of Galois element g, canonical residues,
 * u64[beta][2][L+K][N] (component 0 = b, 1 = a). */
int fheon_key_download(fheon_ctx *ctx, uint64_t galois, uint64_t *host);
/* Install the key of Galois element g (0 = the relinearisation key) from
 * host limbs in the layout fheon_key_download writes: u64[beta][2][L+K][N],
 * canonical residues (the reverse of the download: converted to Montgomery
 * form on the device).  The load half of a key checkpoint (paper Sec. 5.7
 * loads each block's keys from storage).  A key already present is
 * overwritten in place, after the context's queued work, so that graphs
 * captured with it stay valid.  FHEON_ERR_ARG for a bad element or any
 * residue not below its limb's modulus (checked on the host before any
 * copy); blocks until the key is on the device. */
int fheon_key_upload(fheon_ctx *ctx, uint64_t galois, const uint64_t *host);
/* The Galois elements of the resident keys in increasing order (0 is the
 * relinearisation key).  With out == NULL, *n receives the count; else *n
 * is out's capacity on entry (FHEON_ERR_ARG if too small) and the count on
 * return. */
int fheon_key_list(const fheon_ctx *ctx, uint64_t *out, uint32_t *n);
/* Galois element of a slot rotation by r (negative r allowed). */
uint64_t fheon_galois_elt(const fheon_ctx *ctx, int32_t r);

/* ------------------------------------------------------------------ */
/* Plaintexts (paper Sec. 3.2, encoding C^{N/2} -> R)                 */
/* ------------------------------------------------------------------ */
/* Encode n <= N/2 complex slots (re, im; im may be NULL) at `scale` into a
 * plaintext over Q_level: coefficients m_k = round(scale * tau^-1(z)_k)
 * (FP64 special FFT on the device, round half away from zero), then RNS
 * reduction and NTT.  Errors: FHEON_ERR_ARG if a coefficient exceeds 2^62. */
int fheon_encode_plain(fheon_ctx *ctx, const double *re, const double *im, uint32_t n, uint32_t level,
                       double scale, fheon_pt **out);
/* Plaintext from N integer coefficients (host), over Q_level, tagged with
 * `scale`. */
int fheon_plain_from_coeffs(fheon_ctx *ctx, const int64_t *coeffs, uint32_t level, double scale,
                            fheon_pt **out);
/* Blocking: the integer coefficients the device encoder produces for z
 * (same arithmetic as fheon_encode_plain, before RNS reduction). */
int fheon_encode_coeffs(fheon_ctx *ctx, const double *re, const double *im, uint32_t n, double scale,
                        int64_t *coeffs);
/* Blocking decode of a plaintext into n slots (re, im; im may be NULL):
 * INTT, centred lift from the lowest two limbs (exact while |m| < q0*q1/2),
 * FP64 FFT, division by the plaintext's scale. */
int fheon_decode(fheon_ctx *ctx, const fheon_pt *pt, double *re, double *im, uint32_t n);
int fheon_pt_info(const fheon_pt *pt, uint32_t *level, double *scale);
int fheon_pt_download(fheon_ctx *ctx, const fheon_pt *pt, uint64_t *host);
int fheon_pt_destroy(fheon_pt *pt);

/* ------------------------------------------------------------------ */
/* Ciphertexts (paper Sec. 5.7, encryption layer)                       */
/* ------------------------------------------------------------------ */
/* Public-key encryption of pt (must be at level L):
 * ct = (v*b + e0 + m, v*a + e1), v ternary, e0, e1 Gaussian, drawn from
 * streams (seed, 6|7|8, nonce).  fheon_encrypt uses a per-context counter
 * as the nonce. */
int fheon_encrypt(fheon_ctx *ctx, const fheon_pk *pk, const fheon_pt *pt, fheon_ct **out);
int fheon_encrypt_seeded(fheon_ctx *ctx, const fheon_pk *pk, const fheon_pt *pt, uint64_t nonce,
                         fheon_ct **out);
/* m = c0 + c1*s over Q_level, as a plaintext with the ciphertext's scale. */
int fheon_decrypt(fheon_ctx *ctx, const fheon_sk *sk, const fheon_ct *ct, fheon_pt **out);
/* Zero ciphertext at `level` with `scale`, for use as an output buffer. */
int fheon_ct_create(fheon_ctx *ctx, uint32_t level, double scale, fheon_ct **out);
int fheon_ct_destroy(fheon_ct *ct);
int fheon_ct_info(const fheon_ct *ct, uint32_t *level, double *scale);
/* Copy u64[2][level][N] residues from / to host memory on the context's
 * stream.  Upload is asynchronous when `host` is pinned, else it blocks;
 * download blocks.  Residues are not range-checked on upload. */
int fheon_ct_upload(fheon_ctx *ctx, fheon_ct *ct, const uint64_t *host);
int fheon_ct_download(fheon_ctx *ctx, const fheon_ct *ct, uint64_t *host);
/* The same copies queued on `stream` (NULL: the context's stream) without
 * waiting: the host buffer must stay valid (and, for full speed, pinned) until
 * the stream has passed the copy; ordering against the context's work is the
 * caller's (events), so transfers of one batch can overlap the key switching
 * of another. */
/* n ciphertexts at the given levels in one device allocation, back to back
 * (ciphertext i: 2 * levels[i] * N words), zeroed; each handle is destroyed as
 * usual and the allocation goes with the last of them.  A batch moves to and
 * from the host in one copy (below). */
int fheon_ct_create_batch(fheon_ctx *ctx, const uint32_t *levels, uint32_t n, double scale, fheon_ct **out);
/* Copies of n ciphertexts from/to `host` holding them back to back (ciphertext
 * i: 2 * level_i * N words), queued on `stream` (NULL: the context's) without
 * waiting: one copy when they are one batch in order at their created levels,
 * else one copy each.  Host memory as for fheon_ct_upload_async. */
int fheon_ct_upload_many_async(fheon_ctx *ctx, fheon_ct *const *cts, uint32_t n, const uint64_t *host, void *stream);
int fheon_ct_download_many_async(fheon_ctx *ctx, const fheon_ct *const *cts, uint32_t n, uint64_t *host,
                                 void *stream);
int fheon_ct_upload_async(fheon_ctx *ctx, fheon_ct *ct, const uint64_t *host, void *stream);
int fheon_ct_download_async(fheon_ctx *ctx, const fheon_ct *ct, uint64_t *host, void *stream);
/* Device address of the ciphertext's u64[2][level][N] array. */
int fheon_ct_device_ptr(const fheon_ct *ct, void **dptr);

/* ------------------------------------------------------------------ */
/* Homomorphic evaluation                                             */
/* ------------------------------------------------------------------ */
/* Rotation by `step` slots (paper Sec. 3.2 rotation; Alg. 1 Rot_k):
 *   (c0, c1) -> (sigma_g(c0), sigma_g(c1)) in the evaluation domain, then
 *   hybrid key switching of sigma_g(c1) from sigma_g(s) to s: INTT, ModUp
 *   of each digit by fast base conversion, NTT, inner product with the
 *   key, ModDown by P; out = (sigma_g(c0) + ks0, ks1).
 * out is resized to in's level and takes its scale; out may equal in.
 * Errors: FHEON_ERR_NO_KEY if no key for 5^step. */
int fheon_rotate(fheon_ctx *ctx, const fheon_ct *in, int32_t step, fheon_ct *out);
int fheon_rotate_galois(fheon_ctx *ctx, const fheon_ct *in, uint64_t galois, fheon_ct *out);

/* fheon_rotate without any device allocation.  The paper has no counterpart:
 * this serves callers that must not allocate while they rotate -- a server
 * whose device memory is partitioned once at start-up, a latency-critical
 * path that cannot pay for cudaMalloc/cudaFree (cudaFree synchronises the
 * device), or work recorded inside a stream capture, where allocation calls
 * are not permitted.  The result is identical to fheon_rotate.
 *  - The caller passes the input and an output ciphertext that already holds
 *    at least in's level limbs per component (fheon_ct_create); out must not
 *    be in.  FHEON_ERR_ARG otherwise.
 *  - The key-switching workspace is a fixed 32 MiB device array inside the
 *    library (reserved on every GPU that loads it, until the process exits).
 *    A rotation needs (l + beta*(l+K) + 2*(l+K) + 2K + 2l) * N * 8 bytes at
 *    level l (e.g. N = 2^13, L = 3, K = 1: 2 MiB; N = 2^16 with K = 4 and
 *    four limbs per digit fits up to level 5, 29.5 MiB); larger requests fail
 *    with FHEON_ERR_ARG and a message.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.
 *  - All calls share the array and it keeps the last call's contents (a
 *    rotation never reads workspace it did not write first).  Calls that
 *    overlap on the GPU race on it: serialise them on one stream.
 * Errors: as fheon_rotate. */
int fheon_rotate_noalloc(fheon_ctx *ctx, const fheon_ct *in, int32_t step, fheon_ct *out);

/* One batched rotation request: rotate `in` by `step` into `out`. */
typedef struct fheon_rot_item {
    const fheon_ct *in;
    fheon_ct *out;
    int32_t step;
} fheon_rot_item;
/* Rotate many ciphertexts, at any mix of levels and steps, with one launch
 * per pipeline stage over a device work list (instead of one launch
 * sequence per ciphertext).  Bit-identical to n calls of fheon_rotate.
 * Outputs must be distinct from every input of the batch. */
int fheon_rotate_batch(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n);
/* Hoisted rotations, the "fast rotations" the paper's CKKS library provides
 * (Sec. 3.2; Halevi-Shoup hoisting in the hybrid key-switching form):
 * outs[i] = Rot_{steps[i]}(in) for i < n, with one INTT + ModUp + NTT of c1
 * shared by all n.  Rotation i applies sigma_g to the raised digits in the
 * evaluation domain (a gather inside the key inner product), takes the inner
 * product with its own key and its own ModDown, and adds sigma_g(c0).  The
 * results decrypt like fheon_rotate's but differ from them in the low bits
 * for g != 1 (the fast base conversion is not odd).  Outputs must be distinct
 * from `in` and from each other (FHEON_ERR_ARG); a missing key gives
 * FHEON_ERR_NO_KEY before any launch; n = 0 does nothing. */
int fheon_rotate_hoisted(fheon_ctx *ctx, const fheon_ct *in, const int32_t *steps, uint32_t n,
                         fheon_ct *const *outs);
/* fheon_rotate_batch with hoisting: items that share an input pointer share
 * one raising (results as fheon_rotate_hoisted per input). */
int fheon_rotate_batch_hoisted(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n);

/* out = ct * pt slot-wise (paper Sec. 5.1, kernel-vector products); levels
 * must match (the plaintext may be at a higher level: its lowest limbs are
 * used); scale(out) = scale(ct) * scale(pt). */
int fheon_mul_plain(fheon_ctx *ctx, const fheon_ct *ct, const fheon_pt *pt, fheon_ct *out);
/* out = sum_t cts[t] * pts[t] slot-wise (paper Sec. 5.1: the kernel-vector
 * products of a layer and their sum, in one pass): n >= 1 ciphertexts at one
 * level, plaintexts at that level or above, every product at the same scale
 * (1e-9 relative; else FHEON_ERR_SCALE); out is distinct from every input
 * (FHEON_ERR_ARG).  Bit-identical to n fheon_mul_plain calls summed with
 * fheon_add.  scale(out) = the products' scale. */
int fheon_mac_plain(fheon_ctx *ctx, const fheon_ct *const *cts, const fheon_pt *const *pts, uint32_t n,
                    fheon_ct *out);
/* Ciphertext product with relinearisation (the multiplications of the
 * Chebyshev ReLU, paper Alg. 4 and Sec. 5.6): the tensor (a0 b0, a0 b1 + a1 b0,
 * a1 b1) decrypts under (1, s, s^2); its last part is key-switched from s^2 to
 * s on the rotation's key-switching kernels with the relinearisation key.
 * Equal levels (else FHEON_ERR_LEVEL); FHEON_ERR_NO_KEY without
 * fheon_relinkeygen.  scale(out) = scale(a) * scale(b); no rescale.  out may
 * be a or b. */
int fheon_mul_relin(fheon_ctx *ctx, const fheon_ct *a, const fheon_ct *b, fheon_ct *out);
/* out = v * ct for an integer v (exact; scale unchanged). */
int fheon_mul_int(fheon_ctx *ctx, const fheon_ct *ct, int64_t v, fheon_ct *out);
/* out = ct + v, v an integer constant polynomial (every slot gains v / scale). */
int fheon_add_int(fheon_ctx *ctx, const fheon_ct *ct, int64_t v, fheon_ct *out);
/* out = ct + c in every slot: fheon_add_int with v = llround(c * scale(ct))
 * (FHEON_ERR_ARG when |c * scale| >= 2^62). */
int fheon_add_const(fheon_ctx *ctx, const fheon_ct *ct, double c, fheon_ct *out);
/* out = c * ct rescaled once, landing on scale `target`: the ciphertext is
 * multiplied by K = llround(((c * target) * q_{l-1}) / scale(ct)) (binary64,
 * in that order) and rescaled by q_{l-1}; scale(out) = target, level l - 1.
 * Used to scale by constants and to align levels and scales before adding
 * (paper Alg. 4's coefficient products and its 1/beta scaling).
 * FHEON_ERR_LEVEL below level 2, FHEON_ERR_ARG when |K| >= 2^62. */
int fheon_mul_const_rescale(fheon_ctx *ctx, const fheon_ct *ct, double c, double target, fheon_ct *out);
/* out = a + b; equal levels, scales equal to 1e-9 relative, else
 * FHEON_ERR_LEVEL / FHEON_ERR_SCALE. */
int fheon_add(fheon_ctx *ctx, const fheon_ct *a, const fheon_ct *b, fheon_ct *out);
/* out = ct + pt (c0 only). */
int fheon_add_plain(fheon_ctx *ctx, const fheon_ct *ct, const fheon_pt *pt, fheon_ct *out);
/* Floor rescale by the last prime q_t (paper Sec. 6, depth and rescaling):
 * out_i = (x_i - [x]_{q_t}) * q_t^-1 mod q_i, level - 1, scale / q_t. */
int fheon_rescale(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out);
/* Keep the lowest `level` limbs (level <= in's level). */
int fheon_drop_level(fheon_ctx *ctx, const fheon_ct *in, uint32_t level, fheon_ct *out);

/* ------------------------------------------------------------------ */
/* Secure layers (paper Sec. 5)                                       */
/* ------------------------------------------------------------------ */
/* Rotation steps fheon_conv2d needs on a ring of degree N for this shape
 * (host only, no context): for the special convolution (in_ch = out_ch = 1,
 * odd k, stride 1, pad (k-1)/2) di*W + dj for every non-zero tap (di, dj) in
 * [-(k-1)/2, (k-1)/2]^2 (paper Sec. 5.3 and the rotation-index analysis of
 * Sec. 5.7); otherwise the tap steps (x - pad)*W + (y - pad), the block
 * shifts -delta*H*W (delta = f - c != 0) and, when the outputs need
 * compacting, the repack's steps.  Sorted, distinct.  With out == NULL only
 * *n is set (the count); else *n is out's capacity on entry (FHEON_ERR_ARG if
 * too small) and the count on return.  FHEON_ERR_ARG for a zero size, N not
 * a power of two, a kernel larger than the padded input, or maps that do not
 * fit N/2 slots. */
int fheon_conv2d_rotation_steps(uint32_t N, uint32_t in_ch, uint32_t out_ch, uint32_t k, uint32_t stride,
                                uint32_t pad, uint32_t in_h, uint32_t in_w, int32_t *out, uint32_t *n);
/* Prepare a special convolution (paper Sec. 5.3, Alg. 1-3 generalised to
 * odd k): one output channel per layer call, in_ch input channels packed
 * at slot c*H*W + h*W + w, weights w[in_ch][k][k], optional bias.  The
 * tap vectors (weight x boundary mask of Alg. 2/3) are encoded at scale
 * q_{level-1} so that one rescale restores the input scale.
 * stride must be 1 and pad (k-1)/2 (FHEON_ERR_UNIMPLEMENTED otherwise). */
int fheon_conv2d_prepare(fheon_ctx *ctx, uint32_t in_ch, uint32_t k, uint32_t stride, uint32_t pad,
                         uint32_t in_h, uint32_t in_w, const double *w, const double *bias,
                         uint32_t level, double in_scale, fheon_layer **out);
/* Prepare from caller-made tap plaintexts (k*k of them, taps row-major,
 * each over Q_level) and an optional bias plaintext (level-1). */
int fheon_conv2d_prepare_plain(fheon_ctx *ctx, uint32_t in_ch, uint32_t k, uint32_t in_h, uint32_t in_w,
                               uint32_t level, const fheon_pt *const *taps, const fheon_pt *bias,
                               fheon_layer **out);
/* Apply: for each tap, Rot_{di*W+dj}(in) * tap plaintext, summed, one
 * rescale, channel sum by Rot_{H*W} (in_ch > 1), bias added. */
int fheon_conv2d_apply(fheon_ctx *ctx, const fheon_layer *layer, const fheon_ct *in, fheon_ct *out);
/* fheon_conv2d_apply through a CUDA graph.  The first call for a given
 * (input buffer, output buffer, level) runs the layer eagerly, then captures
 * the same launch sequence on the context's stream (which must be a created
 * stream, not the legacy default stream) into a graph kept by the layer;
 * later calls with the same buffers replay it with one cudaGraphLaunch.
 * Results are identical to fheon_conv2d_apply.  The graph holds the buffer
 * addresses it was captured with: rotation keys, the layer and both
 * ciphertexts must stay alive and in place while it is replayed. */
int fheon_conv2d_apply_graph(fheon_ctx *ctx, const fheon_layer *layer, const fheon_ct *in, fheon_ct *out);
/* Convolution in one call (paper Sec. 5.1 equation with padding and stride,
 * Sec. 5.2 output size): the input ciphertext holds the flattened
 * (in_ch, in_h, in_w) map at slot c*H*W + h*W + w (Sec. 5.1 flattening); w is
 * w[out_ch][in_ch][k][k] (row-major, cross-correlation as in Sec. 5.1), bias
 * b[out_ch] or NULL.  The output holds the flattened (out_ch, Ho, Wo) map at
 * f*Ho*Wo + i*Wo + j, Ho = (in_h + 2 pad - k)/stride + 1 (likewise Wo), zero in
 * every other slot.  One output channel from one input channel with odd k,
 * stride 1 and pad (k-1)/2 is the special convolution of Sec. 5.3 (one
 * level); every other shape is the rotation-sum convolution of
 * fheon_conv_prepare on that map (one level), followed, when its outputs are
 * not already compact (stride > 1, or an output smaller than the input), by
 * one repack layer (one more level).  Needs the rotation keys of
 * fheon_conv2d_rotation_steps.  Errors: FHEON_ERR_ARG for zero sizes or maps
 * that do not fit N/2 slots; FHEON_ERR_NO_KEY; FHEON_ERR_LEVEL when the input
 * has too few levels.  Asynchronous on the context's stream. */
int fheon_conv2d(fheon_ctx *ctx, const fheon_ct *in, uint32_t in_ch, uint32_t out_ch, uint32_t k, uint32_t stride,
                 uint32_t pad, uint32_t in_h, uint32_t in_w, const double *w, const double *bias, fheon_ct *out);
int fheon_layer_destroy(fheon_layer *layer);

/* ------------------------------------------------------------------ */
/* Packed network layers on a fheon_map (paper Sec. 5.1, 4.4, 4.5)     */
/* ------------------------------------------------------------------ */
/* Rotation-sum layer from the caller's plaintexts:
 *   x'  = sum_c Rot_{fold[c]}(in)   (nf > 0; the nf rotations hoisted from in)
 *   out = sum_g Rot_{s[g]}( rescale( sum_t Rot_{r[t]}(x') * pts[g*nt + t] ) ) (+ bias)
 * The nt tap rotations (distinct steps; 0 = the input itself) are hoisted
 * from the input; each group's products are summed in one pass and rescaled
 * once; the ng group sums move by one batched rotation (s[g] = 0: none) and are
 * added; bias (optional, level >= level-1) is added last.  pts[g*nt + t] may
 * be NULL (no product); each group needs one.  Plaintexts at `level` or above,
 * encoded at scale q_{level-1}; they stay owned by the caller and must outlive
 * the layer.  Output level: level - 1. */
int fheon_linear_prepare_plain(fheon_ctx *ctx, uint32_t nf, const int32_t *fold, uint32_t nt, const int32_t *r,
                               uint32_t ng, const int32_t *s, const fheon_pt *const *pts, const fheon_pt *bias,
                               uint32_t level, fheon_layer **out);
/* Fully connected layer from the caller's plaintexts (Sec. 5.5): t_k =
 * rescale(in * W[k]) for each of the m neurons; each t_k summed over all N/2
 * slots by rotate-and-add (steps 1, 2, ..., N/4, batched over the neurons);
 * out = rescale(sum_k t_k * E[k]) (+ bias, level >= level-2).  W at `level`
 * (scale q_{level-1}), E at level-1 (scale q_{level-2}).  Output level:
 * level - 2.  Caller-owned plaintexts. */
int fheon_fc_prepare_plain(fheon_ctx *ctx, uint32_t m, const fheon_pt *const *W, const fheon_pt *const *E,
                           const fheon_pt *bias, uint32_t level, fheon_layer **out);
/* Convolution (Sec. 5.1 and Sec. 5.2 equations; zero padding `pad`, stride
 * `stride`) of the map `in` to F output channels, kernel K[F][C][k][k],
 * bias[F] (or NULL): a rotation-sum layer with one group per block shift
 * f - c.  Output (i, j) stays at input-grid position (stride*i, stride*j):
 * the output map has the input's grid and block, dilation dil*stride and
 * (H + 2 pad - k)/stride + 1 rows and columns; the striding costs no
 * rotation and no level.  Plaintexts encoded on the device, owned by the
 * layer.  Output level: level - 1, scale in_scale. */
int fheon_conv_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t F, uint32_t k, uint32_t stride, uint32_t pad,
                       const double *K, const double *bias, uint32_t level, double in_scale, fheon_layer **out);
/* Average pooling (Sec. 5.4): the k x k window sum by k^2 hoisted rotations
 * times one mask of 1/k^2 at the stride-aligned outputs.  The outputs stay in
 * place: the output map's dilation is the input's times `stride`. */
int fheon_avgpool_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t k, uint32_t stride, uint32_t level,
                          fheon_layer **out);
/* Fully connected layer (Sec. 5.5 equation): W[m][C*H*W] over the map's
 * values in (c, i, j) order, bias[m] (or NULL); output: the m neurons in slots
 * [0, m) (map {1, 1, m, m, 1, m}).  A rotation-sum layer in diagonal form:
 * when the channels interleave on the dilation grid (C <= dil^2) they are
 * first folded into block 0 (x' = sum_c Rot_{c*block - off_c}(in)); then
 * y[k] = sum_d diag_d[k] x'[k + d] by baby-step giant-step over the span of
 * d (about 2 sqrt(span) rotations).  Output level: level - 1, scale in_scale. */
int fheon_fc_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t m, const double *W, const double *bias,
                     uint32_t level, double in_scale, fheon_layer **out);
/* Repack a feature map into another layout of the same (C, H, W) in one
 * level (the paper's striding by extraction, Sec. 5.2: the values a strided
 * layer leaves at dilated positions gathered into a compact grid): out =
 * sum_o m_o Rot_o(in), with m_o one at every destination slot whose source is
 * o slots further on, as baby-step/giant-step rotation sums; masks at scale
 * q_{level-1} (the output keeps the input's scale; every slot outside the
 * output map is zero).  At most 1024 distinct shifts (split larger moves
 * into steps). */
int fheon_repack_prepare(fheon_ctx *ctx, const fheon_map *in, const fheon_map *out, uint32_t level,
                         fheon_layer **layer);
/* Global average pooling (Sec. 5.4, used by ResNet): the mean over each
 * channel's whole H x H map, as average pooling with k = stride = H (one
 * value per channel, at the channel's first slot). */
int fheon_global_avgpool_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t level, fheon_layer **out);
/* One-shot layers at ct's level and scale (prepare, apply, release). */
int fheon_avgpool(fheon_ctx *ctx, const fheon_ct *ct, const fheon_map *in, uint32_t k, uint32_t stride, fheon_ct *out);
int fheon_global_avgpool(fheon_ctx *ctx, const fheon_ct *ct, const fheon_map *in, fheon_ct *out);
/* Fully connected layer with the paper's key budget (Sec. 5.5, the number of
 * rotation keys the system keeps): the diagonal form of fheon_fc_prepare when
 * its rotation steps number at most max_keys (0: no limit), else the paper's
 * form (one product per neuron, the slot sum by rotate-and-add with log2(N/2)
 * keys, a one-hot placement; two levels); FHEON_ERR_ARG when max_keys is
 * below log2(N/2). */
int fheon_fc(fheon_ctx *ctx, const fheon_ct *ct, const fheon_map *in, uint32_t m, const double *W, const double *bias,
             uint32_t max_keys, fheon_ct *out);
/* ------------------------------------------------------------------ */
/* CKKS bootstrapping (the paper's "Bootstrapping Layer" among its support
 * functions, placed before the ReLUs of its deeper networks): the published
 * full-slot method of Cheon, Han, Kim, Kim and Song (2018) with the slot
 * transforms factored into the butterfly stages of the special FFT and
 * applied as baby-step/giant-step rotation sums (Chen, Chillotti, Song 2019)
 * and the modular reduction as a scaled cosine plus double-angle steps (Han,
 * Ki 2020).  Steps: ModRaise of limb q_0 into all L primes; CoeffToSlot
 * (cts_levels rotation-sum levels); real and imaginary parts through the
 * conjugation (Galois element 2N - 1); EvalMod on each (the Chebyshev series
 * of cos(2 pi (K x - 1/4) / 2^r), then r doublings c <- 2c^2 - 1);
 * recombination; SlotToCoeff (stc_levels levels).  Consumes
 * cts_levels + ceil(log2 degree) + 1 + doublings + stc_levels levels: a
 * bootstrap of a context with L primes leaves the message at level
 * L minus that.  Inputs are any ciphertext at level >= 1 whose message
 * coefficients are small against q_0 (slots of magnitude <= 1 at a scale
 * 2^10 or more below q_0) and whose scale is the one the layer was prepared
 * for; the output has that scale (to 1e-9) and the same message.  Keys: the
 * layer's rotation steps, the conjugation and the relinearisation key
 * (fheon_bootstrap_keygen makes them all).
 *
 * Sparse bootstrap (slots = n_s <= N/4; OpenFHE, which the paper runs, does
 * the same for a message of fewer than N/2 slots): the input, at level >= 2,
 * is multiplied by the mask of slots [0, n_s) (one level, the mask encoded
 * at scale q_1 so the scale is kept) and repeated in every copy of n_s slots
 * (x + Rot_{n_s 2^j}(x) at level 1), so that its polynomial lies in
 * Z[X^(N / 2 n_s)].  After ModRaise the trace (the same sums at level L)
 * keeps the coefficients of that subring; CoeffToSlot is the n_s-slot
 * transform in every copy and ends in the factor 1 on even copies and -i on
 * odd ones, so that c + conj(c) holds the low coefficients in the even copies
 * and the high ones in the odd copies: ONE EvalMod instead of two.
 * SlotToCoeff starts with the map (a, b) -> a + i b in every copy.  The
 * output holds slots [0, n_s) of the input in every copy of n_s slots.
 * Levels consumed above q_0 are the same as the full bootstrap's. */
typedef struct fheon_boot_params {
    uint32_t cts_levels; /* levels of CoeffToSlot, 1 .. log2(N/2) */
    uint32_t stc_levels; /* levels of SlotToCoeff, 1 .. log2(N/2) */
    uint32_t K;          /* EvalMod's range: |t / q_0| < K for the raised plaintext t */
    uint32_t degree;     /* Chebyshev degree of the cosine */
    uint32_t doublings;  /* double-angle steps r */
    uint32_t baby;       /* baby steps of every BSGS level (0: fewest rotations) */
    uint32_t slots;      /* 0 or N/2: every slot; a power of two in [2, N/4]: the
                          * sparse bootstrap of slots [0, slots) (below) */
    uint32_t unmasked;   /* sparse only, 1: inputs are zero outside slots
                          * [0, slots) (a convolution's output, say), so the
                          * mask is left out and inputs at level 1 are taken */
} fheon_boot_params;
/* Defaults for a context: 3 + 3 levels, K the power of two at or above
 * 8 sqrt(N / 18) (eight standard deviations of t / q_0 for a uniform ternary
 * secret), r = log2 K, degree 27. */
int fheon_boot_params_default(const fheon_ctx *ctx, fheon_boot_params *p);
/* EvalMod's coefficients c_0..c_degree: the Chebyshev interpolant of
 * cos(2 pi (K z - 1/4) / 2^r) at the degree+1 nodes cos(pi (k + 1/2) / (degree + 1)). */
int fheon_evalmod_coeffs(uint32_t K, uint32_t doublings, uint32_t degree, double *out);
/* Prepare a bootstrap (p NULL: the defaults) for inputs of scale in_scale:
 * the merged stage diagonals of both transforms in BSGS form, encoded on the
 * device and owned by the layer.  FHEON_ERR_LEVEL when the context is too
 * shallow.  Apply it with fheon_layer_apply. */
int fheon_bootstrap_prepare(fheon_ctx *ctx, const fheon_boot_params *p, double in_scale, fheon_layer **out);
/* A bootstrap from caller-prepared levels (rotation-sum layers from
 * fheon_linear_prepare_plain, without fold or bias, at levels L, L-1, ... for
 * CoeffToSlot and from L - cts_levels - ceil(log2 degree) - 1 - doublings
 * down for SlotToCoeff) and EvalMod coefficients (degree + 1).  The layer
 * keeps pointers to the levels: they must outlive it. */
int fheon_bootstrap_compose(fheon_ctx *ctx, const fheon_boot_params *p, const fheon_layer *const *cts,
                            const fheon_layer *const *stc, const double *coeffs, double in_scale, fheon_layer **out);
/* Sparse bootstrap: replace the input mask the layer encoded (slots
 * [0, n_s) at level 2, scale q_1) by the caller's plaintext, which must
 * outlive the layer (for checking the layer against an independent encoder).
 * FHEON_ERR_ARG for a full bootstrap or a plaintext below level 2. */
int fheon_bootstrap_set_mask(fheon_ctx *ctx, fheon_layer *layer, const fheon_pt *mask);
/* Generate every key a bootstrap layer uses. */
int fheon_bootstrap_keygen(fheon_ctx *ctx, const fheon_sk *sk, const fheon_layer *layer);
/* Output level and scale of a bootstrap layer (scale 0 for a composed one). */
int fheon_bootstrap_info(const fheon_layer *layer, uint32_t *out_level, double *out_scale);
/* ModRaise alone: limb q_0 of `in` (any level) to coefficients, lifted to
 * (-q_0/2, q_0/2], into all L primes; out at level L with in's scale. */
int fheon_mod_raise(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out);
/* One-shot bootstrap with the default parameters for ct's scale (the layer
 * is prepared on first use and kept with the context); the keys must exist. */
int fheon_bootstrap(fheon_ctx *ctx, const fheon_ct *ct, fheon_ct *out);
/* Apply any prepared layer (conv2d, ReLU, rotation-sum, FC, bootstrap); `in`
 * at the layer's level (a bootstrap: any level), out distinct from in. */
int fheon_layer_apply(fheon_ctx *ctx, const fheon_layer *layer, const fheon_ct *in, fheon_ct *out);
/* The layer on n inputs at once (outputs distinct from every input and each
 * other): a rotation-sum layer runs every input's tap rotations as one
 * hoisted batch and every group shift as one batch, an FC layer the slot
 * sums of all neurons of all inputs together, a ReLU layer the products of
 * every step of all inputs' series together; conv2d and bootstrap layers run
 * per input.  Each output equals the one fheon_layer_apply gives for its input
 * alone, bit for bit. */
int fheon_layer_apply_batch(fheon_ctx *ctx, const fheon_layer *layer, const fheon_ct *const *ins, uint32_t n,
                            fheon_ct *const *outs);
/* fheon_layer_apply replayed as a CUDA graph: the first call for a given
 * (input buffer, output buffer, workspace, input level and scale) runs the
 * layer eagerly, then captures the same launches on the context's stream
 * (which must not be the legacy default stream) into a graph kept by the
 * layer; later calls with the same key launch the graph.  Inputs with a new
 * scale or level get their own graph. */
int fheon_layer_apply_graph(fheon_ctx *ctx, const fheon_layer *layer, const fheon_ct *in, fheon_ct *out);
/* Rotation steps (keys) the layer uses: *n in = capacity of out (out may be
 * NULL to query), *n out = count; FHEON_ERR_ARG when out is too small. */
int fheon_layer_rotation_steps(const fheon_layer *layer, int32_t *out, uint32_t *n);
/* Output map of a conv, pooling or FC layer prepared from a map. */
int fheon_layer_out_map(const fheon_layer *layer, fheon_map *out);

/* Introspection of a prepared layer, so that a caller (or a test) can check
 * what a builder made against an independent construction: its plan and
 * every plaintext it encoded.  Blocking only where a download is.
 * Kinds of layer: */
#define FHEON_LAYER_SPECIAL_CONV 0 /* fheon_conv2d_prepare */
#define FHEON_LAYER_RELU 1         /* fheon_relu_prepare, fheon_cheb_prepare */
#define FHEON_LAYER_ROTSUM 2       /* rotation-sum: conv, pooling, diagonal FC, repack, slot-transform levels */
#define FHEON_LAYER_FC_SLOTSUM 3   /* fheon_fc_prepare_plain, the paper's per-neuron FC */
#define FHEON_LAYER_BOOTSTRAP 4    /* fheon_bootstrap_prepare / _compose */
/* Kind, level (the input level the layer expects; a bootstrap: L) and
 * counts: a rotation-sum layer has nf fold shifts, nt tap steps and ng
 * groups; a slot-sum FC ng neurons; a special conv nt = k^2 taps and ng = 1;
 * a bootstrap nt CoeffToSlot and ng SlotToCoeff levels; others 0.  Any
 * pointer may be NULL. */
int fheon_layer_plan_info(const fheon_layer *layer, uint32_t *kind, uint32_t *level, uint32_t *nf, uint32_t *nt,
                          uint32_t *ng);
/* A rotation-sum layer's fold shifts fold[nf], tap steps r[nt] and group
 * shifts s[ng] (arrays sized from fheon_layer_plan_info; any may be NULL):
 * out = sum_g Rot_{s_g}(rescale(sum_t Rot_{r_t}(x) * P_{g,t})) + bias, with
 * x = sum_c Rot_{fold_c}(in) when nf > 0.  FHEON_ERR_ARG for other kinds. */
int fheon_layer_plan(const fheon_layer *layer, int32_t *fold, int32_t *r, int32_t *s);
/* Borrow one of a layer's plaintexts (valid while the layer lives; the
 * caller must not destroy it); *out = NULL where the layer has none (a
 * group's tap without a product, no bias).  which: */
#define FHEON_PLAIN_PRODUCT 0 /* rotation-sum P_{g,t}; slot-sum FC weights of neuron g (t = 0); special conv tap t */
#define FHEON_PLAIN_PLACE 1   /* slot-sum FC: the one-hot placement of neuron g */
#define FHEON_PLAIN_BIAS 2    /* the bias (g = t = 0) */
#define FHEON_PLAIN_MASK 3    /* ReLU: the 1/beta mask; special conv with C > 1: the block-0 mask */
#define FHEON_PLAIN_MONO 4    /* bootstrap: X^(N/2) where the parts split (g = 0) and join (g = 1) */
#define FHEON_PLAIN_BOOT_MASK 5 /* sparse bootstrap: the input mask of slots [0, n_s) */
/* FHEON_ERR_ARG for an index out of range or a kind without that plaintext. */
int fheon_layer_plain(const fheon_layer *layer, uint32_t which, uint32_t g, uint32_t t, const fheon_pt **out);
/* Level i of a bootstrap layer: CoeffToSlot levels first (i < nt), then
 * SlotToCoeff (rotation-sum layers, borrowed like plaintexts). */
int fheon_layer_sub(const fheon_layer *layer, uint32_t i, const fheon_layer **out);
/* The series coefficients c_0..c_D of a ReLU / Chebyshev layer or of a
 * bootstrap's EvalMod; with out == NULL only *n (the count) is set, else *n
 * is the capacity on entry (FHEON_ERR_ARG if too small). */
int fheon_layer_coeffs(const fheon_layer *layer, double *out, uint32_t *n);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of inference requests                 */
/* ------------------------------------------------------------------ */
/* A model: a program of steps over a request's registers on one context.
 * Register 0 holds the input and, after the last step, the output.  A step
 * writes register dst from:
 *   FHEON_STEP_LAYER: a prepared layer (bootstraps included) applied to src;
 *   FHEON_STEP_ADD:   the lowest `level` limbs of src plus those of src2;
 *   FHEON_STEP_SCALE: c times src, rescaled onto the model's `scale`.
 * The layers stay owned by the caller and must outlive the model and its
 * requests. */
#define FHEON_STEP_LAYER 0u
#define FHEON_STEP_ADD 1u
#define FHEON_STEP_SCALE 2u
typedef struct fheon_step {
    uint32_t op;
    uint32_t src, src2, dst; /* registers */
    uint32_t level;          /* ADD: the operands' common level */
    const fheon_layer *layer;
    double c;                /* SCALE: the constant */
} fheon_step;
int fheon_model_create_program(fheon_ctx *ctx, const fheon_step *steps, uint32_t n, uint32_t nreg, double scale,
                               fheon_model **out);
/* The ordered layers of a network: one layer step per layer on register 0. */
int fheon_model_create(fheon_ctx *ctx, const fheon_layer *const *layers, uint32_t n, fheon_model **out);
/* The model on one input, step by step on the context's stream (returns when
 * the output is complete). */
int fheon_model_run(fheon_ctx *ctx, const fheon_model *model, const fheon_ct *in, fheon_ct *out);
int fheon_model_destroy(fheon_model *model);
/* Device bytes one request of the model adds in flight with its input at
 * `level`: its registers and step buffers, the working ciphertexts one more
 * input adds to each distinct layer of the model (a layer keeps one set per
 * input of the largest batch it has run), and the largest key-switching
 * workspace one input of a layer's batch needs.  Keys are not included (they
 * are resident before serving).  FHEON_ERR_ARG for a level outside [1, L]. */
int fheon_model_footprint(const fheon_model *model, uint32_t level, size_t *bytes);
/* A server for requests of models on any contexts (each context runs its
 * requests on its own stream; ctx is the context errors are reported on).
 * A submitted request is admitted, in arrival order, while fewer than
 * max_active are in flight and the footprints (fheon_model_footprint) of the
 * admitted requests plus its own fit mem_budget bytes (0: no memory limit);
 * a request that does not fit holds back the later requests of its model,
 * not those of other models; with nothing in flight the oldest waiting
 * request is admitted whatever its size. */
int fheon_server_create(fheon_ctx *ctx, uint32_t max_active, size_t mem_budget, fheon_server **out);
int fheon_server_destroy(fheon_server *server);
/* Queue a request: the model on a copy of `in` (taken on the stream now). */
int fheon_server_submit(fheon_server *server, const fheon_model *model, const fheon_ct *in, uint64_t *id);
/* One scheduling step: drop the requests past the admission timeout, admit
 * what fits, then on every context with requests in flight take its oldest
 * request's stage (model, next step) and run that step for every admitted
 * request at that stage (a layer step as one batch, fheon_layer_apply_batch)
 * on the context's stream; the contexts' batches are enqueued one after the
 * other, so they overlap on the device, and then waited for.  *n_done:
 * requests that finished (or were dropped) in this step.  A result equals
 * the model applied to the request's input alone, bit for bit. */
int fheon_server_step(fheon_server *server, uint32_t *n_done);
/* The result of request `id` into out (then the request is forgotten), or
 * FHEON_PENDING while it runs; FHEON_ERR_ARG for an unknown id;
 * FHEON_ERR_TIMEOUT (then forgotten) for a request dropped because it waited
 * longer than the admission timeout. */
int fheon_server_result(fheon_server *server, uint64_t id, fheon_ct *out);
/* Admission timeout: a request still waiting `seconds` after its submission
 * (host clock) is dropped at the next scheduling step, which counts it in
 * *n_done; its result then reports FHEON_ERR_TIMEOUT.  0 (the default): no
 * limit.  FHEON_ERR_ARG for a negative, infinite or NaN value. */
int fheon_server_set_admit_timeout(fheon_server *server, double seconds);
/* Graph replay (on = 1): a layer step the scheduler runs for one request
 * alone runs as the layer's captured CUDA graph (fheon_layer_apply_graph) on
 * that request's buffers.  A request's buffers go back to a pool of its model
 * when its result is taken, and the model's next request takes them, so its
 * steps replay the graphs captured before (launch gaps between a layer's
 * kernels disappear).  Pooled buffers are outside the memory budget.  Every
 * context of the server's models must run on a created stream, not the
 * legacy default stream: FHEON_ERR_ARG here for the contexts of requests
 * already submitted, and from fheon_server_step otherwise.  Off (the
 * default) frees the pool.  Results are the same bits either way. */
int fheon_server_set_graphs(fheon_server *server, int on);
/* Layer steps that ran as graph replays (their first run, which captures,
 * included). */
int fheon_server_graph_replays(const fheon_server *server, uint64_t *replays);
/* Steps taken, the largest batch so far, requests in flight and waiting. */
int fheon_server_stats(const fheon_server *server, uint64_t *steps, uint32_t *max_batch, uint32_t *active,
                       uint32_t *waiting);
/* The largest batch of one model so far, the admissions the memory budget
 * has deferred (each time a request did not fit), and the footprint bytes the
 * admitted requests hold now.  Any pointer may be NULL. */
int fheon_server_model_stats(const fheon_server *server, const fheon_model *model, uint32_t *max_batch,
                             uint64_t *mem_waits, size_t *held);

/* ------------------------------------------------------------------ */
/* Secure ReLU (paper Sec. 5.6, Alg. 4)                               */
/* ------------------------------------------------------------------ */
/* Chebyshev coefficients c_0..c_degree of f(z) = beta * max(0, z) on [-1, 1],
 * interpolated at the degree+1 Chebyshev nodes cos(pi (k + 1/2) / (degree+1))
 * (the zeros of T_{degree+1}; the paper prints the extrema cos(k pi / d)).
 * out: [degree + 1].  The paper's default degree is 59. */
int fheon_relu_coeffs(double beta, uint32_t degree, double *out);
/* A prepared ReLU for inputs at `level`: when beta > 1 the input is first
 * multiplied by Alg. 4's scale mask (1/beta in slots [0, n), 0 elsewhere,
 * encoded at scale q_{level-1}) and rescaled; then the Chebyshev series of
 * f(z) = beta * max(0, z) is evaluated: T_1 = v, T_2h = 2 T_h^2 - 1,
 * T_2h+1 = 2 T_h+1 T_h - T_1 (products with relinearisation, rescaled), each
 * c_d T_d rescaled onto the input's scale at one common level and summed in
 * order of d, c_0 added.  Output: the input's scale, level - (ceil(log2
 * degree) + 1 + [beta > 1]).  Needs the relinearisation key.  FHEON_ERR_LEVEL
 * when the level is too low; FHEON_ERR_ARG for beta <= 0, degree outside
 * [1, 1023] or n > N/2. */
int fheon_relu_prepare(fheon_ctx *ctx, double beta, uint32_t degree, uint32_t n, uint32_t level,
                       fheon_layer **out);
/* The same with the caller's mask plaintext (at `level` or above, scale
 * q_{level-1}; needed when beta > 1), which stays owned by the caller and
 * must outlive the layer. */
int fheon_relu_prepare_plain(fheon_ctx *ctx, double beta, uint32_t degree, const fheon_pt *mask, uint32_t level,
                             fheon_layer **out);
/* A Chebyshev series layer: out = sum_d c_d T_d(in) for an input in [-1, 1]
 * (the evaluation of fheon_relu_apply without the mask; with the
 * coefficients of fheon_relu_coeffs(beta, D) it is Alg. 4's ReLU of an input
 * already scaled by 1/beta).  Depth ceil(log2 degree) + 1; the output keeps
 * the input's scale. */
int fheon_cheb_prepare(fheon_ctx *ctx, const double *coeffs, uint32_t degree, uint32_t level, fheon_layer **out);
/* Levels a Chebyshev series of this degree consumes (fheon_cheb_prepare, and
 * fheon_relu_* without the mask): 6 for degree 59, 5 for 27; 0 for a degree
 * outside [1, 1023]. */
uint32_t fheon_cheb_depth(uint32_t degree);
/* Apply a prepared ReLU; `in` at the layer's level, out distinct from in. */
int fheon_relu_apply(fheon_ctx *ctx, const fheon_layer *layer, const fheon_ct *in, fheon_ct *out);
/* One-shot: prepare at in's level, apply, release. */
int fheon_relu_approx(fheon_ctx *ctx, const fheon_ct *ct, double beta, uint32_t degree, uint32_t n, fheon_ct *out);

/* Failure detection without a fault: one thread waits on a TMA barrier that
 * nothing completes, with the library's bounded wait cut to `polls` polls
 * (1 .. 2^22); the wait gives up and records FHEON_ERR_TIMEOUT in the
 * context's device error word, which the next fheon_sync reports (and
 * clears).  The context stays usable. */
int fheon_selftest_wait(fheon_ctx *ctx, uint32_t polls);

/* ------------------------------------------------------------------ */
/* Instrumentation (no counterpart in the paper)                      */
/* ------------------------------------------------------------------ */
/* Start recording a CUDA event after every kernel this library launches on
 * the context's stream (one open profile per process). */
int fheon_profile_begin(fheon_ctx *ctx);
/* Stop, synchronise, and write into out[cap] a JSON object
 * {"kernel name": [launches, total device ms], ...}; the time of a launch is
 * the gap between its event and the previous one on the stream.
 * FHEON_ERR_ARG if cap is too small. */
int fheon_profile_end(fheon_ctx *ctx, char *out, size_t cap);

/* Measured integer peaks: the rate of one modular step of the rotation's
 * ALU-bound kernels, run alone on every SM at those kernels' occupancy (three
 * 256-thread CTAs per SM), the step in the form those kernels use it, on one
 * of the context's primes of the right class.  Kinds: */
#define FHEON_PEAK_CT_LAZY 0   /* forward butterfly, no conditional subtraction (q < 2^54) */
#define FHEON_PEAK_GS_LAZY 1   /* inverse butterfly, same primes */
#define FHEON_PEAK_CT_HARVEY 2 /* forward butterfly with Harvey's reductions */
#define FHEON_PEAK_GS_HARVEY 3 /* inverse butterfly with Harvey's reductions */
#define FHEON_PEAK_MAC 4       /* 128-bit multiply-accumulate of a base conversion */
#define FHEON_PEAK_KINDS 5
/* Each thread runs `rounds` rounds of 32 steps (a radix-16 round of four
 * butterfly stages with its 15 twiddle reads; or four source words times
 * eight accumulators, each reduced once per round); the fastest of `reps`
 * launches, timed with CUDA events on the context's stream after one
 * untimed launch, gives *per_s = steps per second.  Blocking; allocates a
 * few KiB through the allocator hook.  FHEON_ERR_ARG for an unknown kind,
 * rounds outside [1, 2^20], reps outside [1, 100], N < 256, or a lazy kind
 * on a context without a prime below 2^54. */
int fheon_alu_peak(fheon_ctx *ctx, uint32_t kind, uint32_t rounds, uint32_t reps, double *per_s);

#ifdef __cplusplus
}
#endif
#endif /* FHEON_H */
