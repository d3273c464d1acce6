// internal.h -- context, handles and device tables of libfheon.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "fheon.h"
#include "modarith.cuh"

namespace fheon {

// ------------------------------------------------------------ allocation
// The free half of the allocator that made a block: a block goes back
// through it even if another allocator was installed since.
struct FreeHook {
    fheon_free_fn fn = nullptr; // nullptr: cudaFree
    void *user = nullptr;
};
void *dev_alloc(size_t bytes, cudaStream_t st, FreeHook *hook);
void dev_free(void *p, size_t bytes, cudaStream_t st, const FreeHook &hook);

struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool owned = true; // false: a view into memory someone else releases
    FreeHook hook;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    DevMem(DevMem &&o) noexcept : p(o.p), bytes(o.bytes), st(o.st), owned(o.owned), hook(o.hook)
    {
        o.p = nullptr;
        o.bytes = 0;
        o.owned = true;
    }
    DevMem &operator=(DevMem &&o) noexcept
    {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; st = o.st; owned = o.owned; hook = o.hook;
            o.p = nullptr; o.bytes = 0; o.owned = true;
        }
        return *this;
    }
    ~DevMem() { release(); }
    void view(void *q, size_t n)
    {
        release();
        p = q;
        bytes = n;
        owned = false;
    }
    bool alloc(size_t n, cudaStream_t s)
    {
        release();
        st = s;
        if (n == 0) return true;
        p = dev_alloc(n, s, &hook);
        if (!p) return false;
        bytes = n;
        return true;
    }
    void release()
    {
        if (p && owned) dev_free(p, bytes, st, hook);
        p = nullptr;
        bytes = 0;
        owned = true;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// An NVTX range over a scope: names the library's phases (key-switching
// stages, layers, the bootstrap's steps, server steps) on a profiler's
// timeline, so that ncu --nvtx can select kernels by phase.  A no-op unless
// a tool is attached.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    // end this range and open the next phase's
    void next(const char *name)
    {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// ------------------------------------------------------------ host math
u64 h_mulmod(u64 a, u64 b, u64 m);
u64 h_powmod(u64 b, u64 e, u64 m);
u64 h_invmod(u64 a, u64 m);
bool h_is_prime(u64 n);
u64 h_min_root(u64 q, u32 N);
u64 h_shoup(u64 w, u64 q);                 // floor(w * 2^64 / q)
ModConst h_modconst(u64 q);
bool h_pick_primes(u32 N, const std::vector<u32> &bits, std::vector<u64> &out);
void h_cdt_table(double sigma, int tail, u64 *T);

// ------------------------------------------------------------ device tables
struct Tables {
    DevMem mc;            // ModConst[L+K]
    DevMem tw_fwd;        // ulonglong2[L+K][N]  (psi^brv(i), shoup)
    DevMem tw_inv;        // ulonglong2[L+K][N]  (psi^-brv(i), shoup)
    DevMem ninv;          // ulonglong2[L+K]     N^-1
    DevMem modup_scale;   // ulonglong2[beta][alpha][alpha]   N^-1 * Dhat_i^-1 mod q_i
    DevMem modup_conv;    // u64[beta][alpha][alpha][L+K]     Mont(Dhat_i mod m_t)
    DevMem moddown_scale; // ulonglong2[K]      N^-1 * Phat_k^-1 mod p_k
    DevMem moddown_conv;  // u64[K][L]          Mont(Phat_k mod q_i)
    DevMem pinv;          // ulonglong2[L]      P^-1 mod q_i
    DevMem pmod;          // ulonglong2[L+K]    P mod m_t
    DevMem rescale_inv;   // ulonglong2[L][L]   [t][i] q_t^-1 mod q_i
    DevMem cdt;           // u64[41]
    DevMem fft_w;         // double2[N/2]  exp(2 pi i j / (N/2))
    DevMem fft_zeta;      // double2[N/2]  exp(pi i k / N)
    DevMem slot_perm;     // u32[N/2]      (5^i mod 2N - 1) / 4
};

struct RotKey {
    DevMem mem; // u64[beta][2][L+K][N], Montgomery form
};

} // namespace fheon

struct fheon_ctx {
    u32 N = 0, logN = 0, L = 0, K = 0, dnum = 0, alpha = 0, beta = 0;
    double scale = 0;
    u64 seed = 0;
    cudaStream_t stream = nullptr;
    std::vector<u64> mod;                 // L+K moduli
    std::vector<ModConst> mc;             // host copy
    fheon::Tables tab;
    std::map<u64, fheon::RotKey> keys;    // by Galois element
    fheon::DevMem ws;                     // key-switching workspace
    fheon::DevMem err;                    // int: error a kernel recorded (FHEON_ERR_TIMEOUT), 0 = none
    size_t ws_limbs = 0;
    u64 enc_counter = 0;
    // key-switching schedule bits: 1 = plain second pass + streaming
    // inner-product kernel (else the inner product is fused into the NTT's
    // second pass); 2 = tiled ModUp conversion (one task per digit and tile
    // over all target limbs; alpha <= 4); 4 = tiled ModDown conversion (K <= 4);
    // 8 = the streaming inner product fed by TMA bulk copies (with bit 1)
    int ks_schedule = 9;
    // false: every batched rotation and product runs one ciphertext at a time,
    // each through its own launch sequence and without hoisting (the plain
    // path batched results are compared with; fheon_ctx_set_batching)
    bool batching = true;
    std::string last_error;

    // limbs of the key-switching workspace at level l
    size_t ks_ws_limbs(u32 l) const;
    u32 beta_at(u32 l) const { return (l + alpha - 1) / alpha; }
    size_t limb_bytes() const { return (size_t)N * 8; }
};

struct fheon_sk {
    fheon::DevMem s; // u64[L+K][N] evaluation form, canonical
};
struct fheon_pk {
    fheon::DevMem b; // u64[2][L][N] (b, a), canonical
};
struct fheon_pt {
    fheon::DevMem m; // u64[level][N] evaluation form, canonical
    u32 level = 0;
    double scale = 1.0;
};
struct fheon_ct {
    fheon::DevMem c; // u64[2][level][N]
    std::shared_ptr<fheon::DevMem> block; // a batch allocation c views into (null: c owns its memory)
    u32 level = 0;   // limbs in use
    u32 cap = 0;     // limbs allocated per component
    double scale = 1.0;
    u64 *c0() const { return c.as<u64>(); }
    u64 *c1(u32 N) const { return c.as<u64>() + (size_t)level * N; }
};

namespace fheon {
// error helpers (set ctx->last_error and return code)
int fail(fheon_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(fheon_ctx *ctx, cudaError_t e, const char *where);
#define FHEON_CUDA(ctx, expr)                                  \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return fheon::cuda_fail((ctx), _e, #expr); \
    } while (0)

// make `ct` an allocation for `level` limbs per component (keeps memory when large enough)
int ct_reshape(fheon_ctx *ctx, fheon_ct *ct, u32 level);
int ensure_workspace(fheon_ctx *ctx, size_t limbs);

// ---------------------------------------------------------------- kernels (host launchers)
// NTT over `n` consecutive limbs at `in` (u64[n][N]) into `out`, limb t under modulus
// index mod0 + t (or the Q/P map below), in the evaluation convention of ntt_core.cuh.
cudaError_t ntt_fwd_limbs(fheon_ctx *ctx, const u64 *in, u64 *out, u32 n, u32 level, u32 first_limb,
                          cudaStream_t st);
cudaError_t ntt_inv_limbs(fheon_ctx *ctx, const u64 *in, u64 *out, u32 n, u32 level, u32 first_limb,
                          cudaStream_t st);

// key switching / rotation (keyswitch.cu)
// The rotation pipeline on caller-provided workspace (ks_ws_limbs(l) limbs);
// launches kernels only, allocates nothing.
// c1add (optional): u64[l][N] added to the key-switched component 1
// (relinearisation: d1; rotation: none)
int keyswitch_rotate(fheon_ctx *ctx, const u64 *c0, const u64 *c1, u32 l, u64 g, const u64 *key, u64 *ws, u64 *out,
                     const u64 *c1add = nullptr);
int rotate_one(fheon_ctx *ctx, const fheon_ct *in, u64 g, fheon_ct *out);
void drop_plans(fheon_ctx *ctx); // release the cached batch plans of a context
void boot_release(const fheon_ctx *ctx); // release the one-shot bootstrap layer of a context
// hoist: items with the same input share one raising of c1 (fast rotations).
// keep (optional) receives a reference to the device plan the launches read,
// for callers that capture them into a graph.
using PlanKeep = std::vector<std::shared_ptr<void>>;
int rotate_many(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n, bool hoist = false, PlanKeep *keep = nullptr);
// one key switch of a batch: input components c0, c1 (u64[level][N] each;
// c1 is switched, c0 joins component 0 of the output), optional c1add joined
// to component 1, output u64[2][level][N], key and Galois element (1: none);
// lead = the item whose raised digits this one reads (itself when it raises)
struct KsItem {
    const u64 *c0 = nullptr, *c1 = nullptr, *c1add = nullptr;
    u64 *out = nullptr;
    const u64 *key = nullptr;
    u64 g = 1;
    u32 level = 0, lead = 0;
};
int ks_many(fheon_ctx *ctx, const KsItem *items, uint32_t n, bool hoist, PlanKeep *keep = nullptr);
// ciphertext products with relinearisation as one batch: out = a * b (lowest
// `level` limbs of each, doubled when `twice`), no rescale; outputs distinct
// from every input
struct RelinItem {
    const fheon_ct *a = nullptr, *b = nullptr;
    u32 level = 0;
    bool twice = false;
    fheon_ct *out = nullptr;
};
int mul_relin_many(fheon_ctx *ctx, const RelinItem *items, uint32_t n, PlanKeep *keep = nullptr);
int rotate_hoisted(fheon_ctx *ctx, const fheon_ct *in, const int32_t *steps, uint32_t n, fheon_ct *const *outs,
                   PlanKeep *keep = nullptr);

// pointwise and rescale (arith.cu)
cudaError_t k_mul_plain(fheon_ctx *ctx, const u64 *ct, const u64 *pt, u64 *out, u32 level, u32 ct_level_out_stride);
// out = sum_t cts[t] * pts[t] (ciphertexts u64[2][level][N], plaintexts' lowest
// level limbs); out must not alias an input when n > MAC_MAX
constexpr u32 MAC_MAX = 32;
cudaError_t k_mac_plain(fheon_ctx *ctx, const u64 *const *cts, const u64 *const *pts, u32 n, u64 *out, u32 level);
// the sums of several groups over one set of taps: outs[g] = sum_t cts[t] *
// pts[g * nt + t] (null plaintexts skipped; every group at least one), all
// ciphertexts u64[2][level][N]; the warps of a block sum MACG_BLOCK_GROUPS
// groups over the same coefficients, so each tap crosses HBM about once per
// that many groups.  Bit-identical to k_mac_plain per group.  nt <=
// MACG_TAPS, ng <= MACG_GROUPS; outputs distinct from the taps
constexpr u32 MACG_TAPS = 64, MACG_GROUPS = 32, MACG_BLOCK_GROUPS = 4;
cudaError_t k_mac_groups(fheon_ctx *ctx, const u64 *const *cts, u32 nt, const u64 *const *pts, u32 ng,
                         u64 *const *outs, u32 level);
cudaError_t k_add(fheon_ctx *ctx, const u64 *a, const u64 *b, u64 *out, u32 nlimb_per_comp, u32 ncomp);
// d = (a0 b0, a0 b1 + a1 b0, a1 b1) (doubled when `twice`) over the lowest
// `level` limbs of each component: u64[3][level][N]
cudaError_t k_tensor(fheon_ctx *ctx, const u64 *a0, const u64 *a1, const u64 *b0, const u64 *b1, u64 *d, u32 level,
                     bool twice = false);
// out = v * ct over `ncomp` components of `level` limbs (input component c at
// ct + c * in_stride; 0 = level * N); out = ct + v on component 0 only
cudaError_t k_mul_int(fheon_ctx *ctx, const u64 *ct, int64_t v, u64 *out, u32 level, u32 ncomp, u64 in_stride = 0);
// ciphertext product with relinearisation of the lowest `level` limbs of a and
// b (either may be at a higher level), doubled when `twice`; no rescale
int mul_relin_at(fheon_ctx *ctx, const fheon_ct *a, const fheon_ct *b, u32 level, bool twice, fheon_ct *out);
// llround(x) into *v when x is finite and |x| < 2^62
bool round_int(double x, int64_t *v);
// c * (the lowest `level` limbs of ct), rescaled onto scale `target`
int mul_const_rescale_at(fheon_ctx *ctx, const fheon_ct *ct, u32 level, double c, double target, fheon_ct *out);
cudaError_t k_add_int(fheon_ctx *ctx, const u64 *ct, int64_t v, u64 *out, u32 level);
// out = sum_t K[t] * (lowest `level` limbs of each component of cts[t], whose
// components sit strides[t] words apart), both components
cudaError_t k_lincomb(fheon_ctx *ctx, const u64 *const *cts, const u64 *strides, const int64_t *K, u32 n, u64 *out,
                      u32 level);
cudaError_t k_add_plain(fheon_ctx *ctx, const u64 *ct, const u64 *pt, u64 *out, u32 level);
int rescale_ct(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out);
// ModRaise: the lowest limb (q_0) of `in`, centred, into all L primes (out at level L)
int mod_raise_ct(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out);
cudaError_t k_decrypt(fheon_ctx *ctx, const u64 *ct, const u64 *s, u64 *m, u32 level);

// sampler / keygen / encrypt (sampler.cu)
int keygen_dev(fheon_ctx *ctx, fheon_sk *sk, fheon_pk *pk);
// key-switching key to s from sigma_g(s) (rotation), or from s^2 when g = 0
// (relinearisation); the sampler streams are tagged g
int galois_key_dev(fheon_ctx *ctx, const fheon_sk *sk, u64 g, RotKey &key);
int encrypt_dev(fheon_ctx *ctx, const fheon_pk *pk, const fheon_pt *pt, u64 nonce, fheon_ct *out);
int plain_from_coeffs_dev(fheon_ctx *ctx, const int64_t *host_coeffs, u32 level, fheon_pt *pt);
// device signed coefficients (N) -> evaluation-form residues over limbs 0..level-1
int limbs_from_coeffs_dev(fheon_ctx *ctx, const long long *dev_coeffs, u32 level, u64 *out);
cudaError_t key_from_mont(fheon_ctx *ctx, const u64 *in, u64 *out, size_t limbs_per_block, u32 blocks);
cudaError_t key_to_mont(fheon_ctx *ctx, u64 *x, size_t limbs_per_block, u32 blocks);

// encoding (encode.cu)
int build_fft_tables(fheon_ctx *ctx);
int encode_dev(fheon_ctx *ctx, const double *re, const double *im, u32 n, double scale, u32 level,
               fheon_pt *pt, int64_t *host_coeffs_out);
int decode_dev(fheon_ctx *ctx, const fheon_pt *pt, double *re, double *im, u32 n);
} // namespace fheon
