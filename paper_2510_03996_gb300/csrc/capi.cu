// capi.cu -- the extern "C" surface of libfheon: allocator hook, errors,
// context creation (constant tables), handles, and dispatch to the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

using namespace fheon;

// ------------------------------------------------------------------ allocator
namespace {
std::mutex g_alloc_mu;
fheon_alloc_fn g_alloc = nullptr;
fheon_free_fn g_free = nullptr;
void *g_alloc_user = nullptr;
}

namespace fheon {
void *dev_alloc(size_t bytes, cudaStream_t st, FreeHook *hook)
{
    fheon_alloc_fn a;
    void *u;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        u = g_alloc_user;
        hook->fn = g_free;
        hook->user = u;
    }
    if (a) return a(bytes, (void *)st, u);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void dev_free(void *p, size_t bytes, cudaStream_t st, const FreeHook &hook)
{
    if (hook.fn) hook.fn(p, bytes, (void *)st, hook.user);
    else cudaFree(p);
}

int fail(fheon_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return code;
}
int cuda_fail(fheon_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, e == cudaErrorMemoryAllocation ? FHEON_ERR_OOM : FHEON_ERR_CUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

int ct_reshape(fheon_ctx *ctx, fheon_ct *ct, u32 level)
{
    if (ct->cap >= level && ct->c.p) {
        ct->level = level;
        return FHEON_OK;
    }
    if (!ct->c.alloc((size_t)2 * level * ctx->N * 8, ctx->stream))
        return fail(ctx, FHEON_ERR_OOM, "ciphertext allocation of %u limbs failed", 2 * level);
    ct->block.reset(); // its own memory now, not a view into a batch
    ct->cap = level;
    ct->level = level;
    return FHEON_OK;
}

int ensure_workspace(fheon_ctx *ctx, size_t limbs)
{
    if (ctx->ws_limbs >= limbs) return FHEON_OK;
    if (!ctx->ws.alloc(limbs * ctx->limb_bytes(), ctx->stream))
        return fail(ctx, FHEON_ERR_OOM, "workspace of %zu limbs failed", limbs);
    ctx->ws_limbs = limbs;
    return FHEON_OK;
}
} // namespace fheon

size_t fheon_ctx::ks_ws_limbs(u32 l) const
{
    const size_t b = beta_at(l);
    return (size_t)l + b * (l + K) + 2 * (size_t)(l + K) + 2 * (size_t)K + 2 * (size_t)l;
}

extern "C" {

const char *fheon_error_string(int code)
{
    switch (code) {
    case FHEON_OK: return "ok";
    case FHEON_ERR_ARG: return "invalid argument";
    case FHEON_ERR_OOM: return "device allocation failed";
    case FHEON_ERR_NO_KEY: return "rotation key missing";
    case FHEON_ERR_LEVEL: return "level mismatch";
    case FHEON_ERR_SCALE: return "scale mismatch";
    case FHEON_ERR_TIMEOUT: return "device wait timed out";
    case FHEON_ERR_CUDA: return "CUDA runtime error";
    case FHEON_ERR_UNIMPLEMENTED: return "not implemented";
    default: return "unknown error";
    }
}

const char *fheon_last_error(const fheon_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int fheon_set_allocator(fheon_alloc_fn alloc, fheon_free_fn free_fn, void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return FHEON_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = user;
    return FHEON_OK;
}

// ------------------------------------------------------------------ parameters (host only)
int fheon_pick_primes(uint32_t N, const uint32_t *bits, uint32_t n, uint64_t *out)
{
    if (!bits || !out || !n || N < 1024 || N > (1u << 17) || (N & (N - 1))) return FHEON_ERR_ARG;
    std::vector<u32> b(bits, bits + n);
    std::vector<u64> m;
    if (!h_pick_primes(N, b, m)) return FHEON_ERR_ARG;
    for (u32 i = 0; i < n; i++) out[i] = m[i];
    return FHEON_OK;
}

uint64_t fheon_min_root(uint64_t q, uint32_t N)
{
    // the search below ends only for a prime q = 1 mod 2N
    if (N < 2 || (N & (N - 1)) || q < 3 || q % (2ull * N) != 1 || !h_is_prime(q)) return 0;
    return h_min_root(q, N);
}

int fheon_gaussian_cdt(uint64_t *out, uint32_t n)
{
    if (!out || n != 41) return FHEON_ERR_ARG;
    u64 T[41];
    h_cdt_table(3.2, 20, T);
    for (u32 i = 0; i < 41; i++) out[i] = T[i];
    return FHEON_OK;
}

// ------------------------------------------------------------------ context
static int upload(fheon_ctx *ctx, DevMem &m, const void *host, size_t bytes)
{
    if (!m.alloc(bytes, ctx->stream)) return fail(ctx, FHEON_ERR_OOM, "table allocation failed");
    FHEON_CUDA(ctx, cudaMemcpyAsync(m.p, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    FHEON_CUDA(ctx, cudaStreamSynchronize(ctx->stream)); // host staging buffers are freed on return
    return FHEON_OK;
}

static int build_tables(fheon_ctx *ctx)
{
    const u32 N = ctx->N, L = ctx->L, K = ctx->K, A = ctx->alpha, B = ctx->beta, n = L + K;
    const u64 *m = ctx->mod.data();
    int rc;
    // NTT twiddles
    std::vector<ulonglong2> fw((size_t)n * N), iv((size_t)n * N);
    std::vector<ulonglong2> ninv(n);
    std::vector<u64> pw(N), pwi(N);
    for (u32 i = 0; i < n; i++) {
        const u64 q = m[i], psi = h_min_root(q, N), psii = h_invmod(psi, q);
        pw[0] = pwi[0] = 1;
        for (u32 e = 1; e < N; e++) {
            pw[e] = h_mulmod(pw[e - 1], psi, q);
            pwi[e] = h_mulmod(pwi[e - 1], psii, q);
        }
        for (u32 k = 0; k < N; k++) {
            u32 r = 0;
            for (u32 b = 0; b < ctx->logN; b++) r |= ((k >> b) & 1u) << (ctx->logN - 1 - b);
            fw[(size_t)i * N + k] = make_ulonglong2(pw[r], h_shoup(pw[r], q));
            iv[(size_t)i * N + k] = make_ulonglong2(pwi[r], h_shoup(pwi[r], q));
        }
        const u64 ni = h_invmod(N % q, q);
        ninv[i] = make_ulonglong2(ni, h_shoup(ni, q));
    }
    if ((rc = upload(ctx, ctx->tab.mc, ctx->mc.data(), sizeof(ModConst) * n))) return rc;
    if ((rc = upload(ctx, ctx->tab.tw_fwd, fw.data(), fw.size() * sizeof(ulonglong2)))) return rc;
    if ((rc = upload(ctx, ctx->tab.tw_inv, iv.data(), iv.size() * sizeof(ulonglong2)))) return rc;
    if ((rc = upload(ctx, ctx->tab.ninv, ninv.data(), ninv.size() * sizeof(ulonglong2)))) return rc;

    auto mont = [&](u64 x, u32 t) { return h_mulmod(x % m[t], ctx->mc[t].r1, m[t]); };
    // ModUp: digit j of size d (its limbs j*A .. j*A+d-1)
    std::vector<ulonglong2> us((size_t)B * A * A, make_ulonglong2(0, 0));
    std::vector<u64> uc((size_t)B * A * A * n, 0);
    for (u32 j = 0; j < B; j++)
        for (u32 d = 1; d <= A; d++) {
            if (j * A + d > L) break;
            for (u32 il = 0; il < d; il++) {
                const u32 i = j * A + il;
                u64 dh = 1;
                for (u32 k = 0; k < d; k++)
                    if (k != il) dh = h_mulmod(dh, m[j * A + k] % m[i], m[i]);
                const u64 sc = h_mulmod(h_invmod(dh, m[i]), ninv[i].x, m[i]);
                us[((size_t)j * A + (d - 1)) * A + il] = make_ulonglong2(sc, h_shoup(sc, m[i]));
                for (u32 t = 0; t < n; t++) {
                    u64 v = 1;
                    for (u32 k = 0; k < d; k++)
                        if (k != il) v = h_mulmod(v, m[j * A + k] % m[t], m[t]);
                    uc[(((size_t)j * A + (d - 1)) * A + il) * n + t] = mont(v, t);
                }
            }
        }
    if ((rc = upload(ctx, ctx->tab.modup_scale, us.data(), us.size() * sizeof(ulonglong2)))) return rc;
    if ((rc = upload(ctx, ctx->tab.modup_conv, uc.data(), uc.size() * sizeof(u64)))) return rc;

    // ModDown
    std::vector<ulonglong2> ds(K), pinv(L), pmod(n);
    std::vector<u64> dc((size_t)K * L);
    for (u32 k = 0; k < K; k++) {
        const u32 pk = L + k;
        u64 ph = 1;
        for (u32 k2 = 0; k2 < K; k2++)
            if (k2 != k) ph = h_mulmod(ph, m[L + k2] % m[pk], m[pk]);
        const u64 sc = h_mulmod(h_invmod(ph, m[pk]), ninv[pk].x, m[pk]);
        ds[k] = make_ulonglong2(sc, h_shoup(sc, m[pk]));
        for (u32 i = 0; i < L; i++) {
            u64 v = 1;
            for (u32 k2 = 0; k2 < K; k2++)
                if (k2 != k) v = h_mulmod(v, m[L + k2] % m[i], m[i]);
            dc[(size_t)k * L + i] = mont(v, i);
        }
    }
    for (u32 t = 0; t < n; t++) {
        u64 P = 1;
        for (u32 k = 0; k < K; k++) P = h_mulmod(P, m[L + k] % m[t], m[t]);
        pmod[t] = make_ulonglong2(P, h_shoup(P, m[t]));
        if (t < L) {
            const u64 pi = h_invmod(P, m[t]);
            pinv[t] = make_ulonglong2(pi, h_shoup(pi, m[t]));
        }
    }
    if ((rc = upload(ctx, ctx->tab.moddown_scale, ds.data(), ds.size() * sizeof(ulonglong2)))) return rc;
    if ((rc = upload(ctx, ctx->tab.moddown_conv, dc.data(), dc.size() * sizeof(u64)))) return rc;
    if ((rc = upload(ctx, ctx->tab.pinv, pinv.data(), pinv.size() * sizeof(ulonglong2)))) return rc;
    if ((rc = upload(ctx, ctx->tab.pmod, pmod.data(), pmod.size() * sizeof(ulonglong2)))) return rc;

    // rescale: [t][i] = q_t^-1 mod q_i
    std::vector<ulonglong2> ri((size_t)L * L, make_ulonglong2(0, 0));
    for (u32 t = 1; t < L; t++)
        for (u32 i = 0; i < t; i++) {
            const u64 v = h_invmod(m[t] % m[i], m[i]);
            ri[(size_t)t * L + i] = make_ulonglong2(v, h_shoup(v, m[i]));
        }
    if ((rc = upload(ctx, ctx->tab.rescale_inv, ri.data(), ri.size() * sizeof(ulonglong2)))) return rc;

    u64 cdt[41];
    h_cdt_table(3.2, 20, cdt);
    if ((rc = upload(ctx, ctx->tab.cdt, cdt, sizeof cdt))) return rc;
    const int no_error = 0;
    if ((rc = upload(ctx, ctx->err, &no_error, sizeof no_error))) return rc;
    return build_fft_tables(ctx);
}

static int ctx_create_impl(u32 N, std::vector<u64> mods, u32 nq, u32 np, u32 dnum, double scale, u64 seed,
                           void *stream, fheon_ctx **out)
{
    if (!out) return FHEON_ERR_ARG;
    *out = nullptr;
    u32 logN = 0;
    while ((1u << logN) < N) logN++;
    if ((1u << logN) != N || logN < 10 || logN > 17) return FHEON_ERR_ARG;
    if (nq < 1 || np < 1 || np > 16 || dnum < 1 || dnum > nq) return FHEON_ERR_ARG;
    const u32 alpha = (nq + dnum - 1) / dnum, beta = (nq + alpha - 1) / alpha;
    if (alpha > 16 || beta > 16) return FHEON_ERR_ARG;
    u64 qmax = 0;
    for (size_t i = 0; i < mods.size(); i++) {
        const u64 q = mods[i];
        if (q >= (1ull << 61) || q % (2ull * N) != 1 || !h_is_prime(q)) return FHEON_ERR_ARG;
        for (size_t k = 0; k < i; k++)
            if (mods[k] == q) return FHEON_ERR_ARG;
        qmax = q > qmax ? q : qmax;
    }
    // lazy accumulations of up to 16 products of residues < qmax reduce by one REDC
    if ((unsigned __int128)qmax * 16 >= ((unsigned __int128)1 << 64)) return FHEON_ERR_ARG;
    fheon_ctx *ctx = new fheon_ctx();
    ctx->N = N;
    ctx->logN = logN;
    ctx->L = nq;
    ctx->K = np;
    ctx->dnum = dnum;
    ctx->alpha = alpha;
    ctx->beta = beta;
    ctx->ks_schedule = 9; // fastest measured default; fheon_autotune_schedule picks per batch
    ctx->scale = scale;
    ctx->seed = seed;
    ctx->stream = (cudaStream_t)stream;
    ctx->mod = mods;
    for (u64 q : mods) ctx->mc.push_back(h_modconst(q));
    int rc = build_tables(ctx);
    if (rc) {
        delete ctx;
        return rc;
    }
    *out = ctx;
    return FHEON_OK;
}

int fheon_ctx_create(uint32_t N, const uint64_t *q, uint32_t nq, const uint64_t *p, uint32_t np, uint32_t dnum,
                     double scale, uint64_t seed, void *stream, fheon_ctx **out)
{
    if (!q || !p) return FHEON_ERR_ARG;
    std::vector<u64> mods(q, q + nq);
    mods.insert(mods.end(), p, p + np);
    return ctx_create_impl(N, mods, nq, np, dnum, scale, seed, stream, out);
}

int fheon_ctx_create_bits(uint32_t N, const uint32_t *qbits, uint32_t nq, const uint32_t *pbits, uint32_t np,
                          uint32_t dnum, double scale, uint64_t seed, void *stream, fheon_ctx **out)
{
    if (!qbits || !pbits || N < 1024 || N > (1u << 17)) return FHEON_ERR_ARG;
    std::vector<u32> bits(qbits, qbits + nq);
    bits.insert(bits.end(), pbits, pbits + np);
    std::vector<u64> mods;
    if (!h_pick_primes(N, bits, mods)) return FHEON_ERR_ARG;
    return ctx_create_impl(N, mods, nq, np, dnum, scale, seed, stream, out);
}

int fheon_ctx_destroy(fheon_ctx *ctx)
{
    if (!ctx) return FHEON_OK;
    cudaStreamSynchronize(ctx->stream);
    boot_release(ctx);
    drop_plans(ctx);
    delete ctx;
    return FHEON_OK;
}

int fheon_ctx_info(const fheon_ctx *ctx, uint32_t *N, uint32_t *L, uint32_t *K, uint32_t *alpha, uint32_t *beta)
{
    if (!ctx) return FHEON_ERR_ARG;
    if (N) *N = ctx->N;
    if (L) *L = ctx->L;
    if (K) *K = ctx->K;
    if (alpha) *alpha = ctx->alpha;
    if (beta) *beta = ctx->beta;
    return FHEON_OK;
}

int fheon_ctx_moduli(const fheon_ctx *ctx, uint64_t *out)
{
    if (!ctx || !out) return FHEON_ERR_ARG;
    memcpy(out, ctx->mod.data(), ctx->mod.size() * sizeof(u64));
    return FHEON_OK;
}

int fheon_ctx_set_stream(fheon_ctx *ctx, void *stream)
{
    if (!ctx) return FHEON_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return FHEON_OK;
}

int fheon_ctx_get_schedule(const fheon_ctx *ctx, int *schedule)
{
    if (!ctx || !schedule) return FHEON_ERR_ARG;
    *schedule = ctx->ks_schedule;
    return FHEON_OK;
}

int fheon_ctx_set_schedule(fheon_ctx *ctx, int schedule)
{
    if (!ctx || schedule < 0 || schedule >= FHEON_NUM_SCHEDULES) return FHEON_ERR_ARG;
    if ((schedule & 8) && !(schedule & 1)) return fail(ctx, FHEON_ERR_ARG, "bulk-copy inner product needs bit 1");
    if ((schedule & 16) && !(schedule & 1)) return fail(ctx, FHEON_ERR_ARG, "radix-8 row passes need bit 1");
    if ((schedule & 2) && ctx->alpha > 4) return fail(ctx, FHEON_ERR_ARG, "tiled ModUp needs alpha <= 4");
    if ((schedule & 4) && ctx->K > 4) return fail(ctx, FHEON_ERR_ARG, "tiled ModDown needs K <= 4");
    ctx->ks_schedule = schedule;
    return FHEON_OK;
}

int fheon_ctx_set_batching(fheon_ctx *ctx, int on)
{
    if (!ctx || (on != 0 && on != 1)) return FHEON_ERR_ARG;
    ctx->batching = on != 0;
    return FHEON_OK;
}

int fheon_autotune_schedule(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n, uint32_t reps, int *best,
                            double *ms_per_batch)
{
    if (!ctx || !items || n == 0 || reps == 0 || !best) return FHEON_ERR_ARG;
    const int old = ctx->ks_schedule;
    cudaEvent_t e0, e1;
    FHEON_CUDA(ctx, cudaEventCreate(&e0));
    FHEON_CUDA(ctx, cudaEventCreate(&e1));
    int pick = -1;
    double pick_ms = 0;
    int rc = FHEON_OK;
    for (int s = 0; s < FHEON_NUM_SCHEDULES && rc == FHEON_OK; s++) {
        if (ms_per_batch) ms_per_batch[s] = -1.0;
        if (fheon_ctx_set_schedule(ctx, s) != FHEON_OK) continue;
        if ((rc = rotate_many(ctx, items, n))) break; // untimed: plans, workspace, caches
        cudaEventRecord(e0, ctx->stream);
        for (uint32_t r = 0; r < reps && rc == FHEON_OK; r++) rc = rotate_many(ctx, items, n);
        cudaEventRecord(e1, ctx->stream);
        if (rc) break;
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) { rc = cuda_fail(ctx, ce, "autotune"); break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / reps;
        if (ms_per_batch) ms_per_batch[s] = per;
        if (pick < 0 || per < pick_ms) { pick = s; pick_ms = per; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->ks_schedule = (rc == FHEON_OK && pick >= 0) ? pick : old;
    if (rc) return rc;
    *best = ctx->ks_schedule;
    return FHEON_OK;
}

// after a synchronisation: the error a kernel recorded since the last check
// (a bounded device wait that gave up), cleared once reported
static int device_error(fheon_ctx *ctx)
{
    int e = 0;
    FHEON_CUDA(ctx, cudaMemcpy(&e, ctx->err.p, sizeof e, cudaMemcpyDeviceToHost));
    if (e == 0) return FHEON_OK;
    const int zero = 0;
    FHEON_CUDA(ctx, cudaMemcpy(ctx->err.p, &zero, sizeof zero, cudaMemcpyHostToDevice));
    return fail(ctx, e, "a kernel's bounded wait ran out; its outputs are not valid");
}

int fheon_sync(fheon_ctx *ctx)
{
    if (!ctx) return FHEON_ERR_ARG;
    FHEON_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return device_error(ctx);
}

// ------------------------------------------------------------------ keys
int fheon_keygen(fheon_ctx *ctx, fheon_sk **sk, fheon_pk **pk)
{
    if (!ctx || !sk || !pk) return FHEON_ERR_ARG;
    fheon_sk *s = new fheon_sk();
    fheon_pk *p = new fheon_pk();
    int rc = keygen_dev(ctx, s, p);
    if (rc) {
        delete s;
        delete p;
        return rc;
    }
    *sk = s;
    *pk = p;
    return FHEON_OK;
}
int fheon_sk_destroy(fheon_sk *sk) { delete sk; return FHEON_OK; }
int fheon_pk_destroy(fheon_pk *pk) { delete pk; return FHEON_OK; }

static int download(fheon_ctx *ctx, const void *dev, void *host, size_t bytes)
{
    FHEON_CUDA(ctx, cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    FHEON_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return device_error(ctx);
}

int fheon_sk_download(fheon_ctx *ctx, const fheon_sk *sk, uint64_t *host)
{
    if (!ctx || !sk || !host) return FHEON_ERR_ARG;
    return download(ctx, sk->s.p, host, (size_t)(ctx->L + ctx->K) * ctx->limb_bytes());
}
int fheon_pk_download(fheon_ctx *ctx, const fheon_pk *pk, uint64_t *host)
{
    if (!ctx || !pk || !host) return FHEON_ERR_ARG;
    return download(ctx, pk->b.p, host, (size_t)2 * ctx->L * ctx->limb_bytes());
}

uint64_t fheon_galois_elt(const fheon_ctx *ctx, int32_t r)
{
    if (!ctx) return 0;
    const int64_t n = ctx->N / 2;
    int64_t e = ((int64_t)r % n + n) % n;
    return h_powmod(5, (u64)e, 2ull * ctx->N);
}

int fheon_galois_keygen(fheon_ctx *ctx, const fheon_sk *sk, const uint64_t *galois, uint32_t n)
{
    if (!ctx || !sk || (n && !galois)) return FHEON_ERR_ARG;
    for (u32 i = 0; i < n; i++) {
        const u64 g = galois[i];
        if ((g & 1) == 0 || g >= 2ull * ctx->N) return fail(ctx, FHEON_ERR_ARG, "bad Galois element %llu", g);
        if (ctx->keys.count(g)) continue;
        RotKey key;
        int rc = galois_key_dev(ctx, sk, g, key);
        if (rc) return rc;
        ctx->keys.emplace(g, std::move(key));
    }
    return FHEON_OK;
}

int fheon_relinkeygen(fheon_ctx *ctx, const fheon_sk *sk)
{
    if (!ctx || !sk) return FHEON_ERR_ARG;
    if (ctx->keys.count(0)) return FHEON_OK;
    RotKey key;
    int rc = galois_key_dev(ctx, sk, 0, key);
    if (rc) return rc;
    ctx->keys.emplace(0, std::move(key));
    return FHEON_OK;
}

int fheon_rotkeygen(fheon_ctx *ctx, const fheon_sk *sk, const int32_t *steps, uint32_t n)
{
    if (!ctx || !sk || (n && !steps)) return FHEON_ERR_ARG;
    std::vector<uint64_t> gs(n);
    for (u32 i = 0; i < n; i++) gs[i] = fheon_galois_elt(ctx, steps[i]);
    return fheon_galois_keygen(ctx, sk, gs.data(), n);
}

int fheon_key_erase(fheon_ctx *ctx, uint64_t galois)
{
    if (!ctx) return FHEON_ERR_ARG;
    auto it = ctx->keys.find(galois);
    if (it == ctx->keys.end()) return fail(ctx, FHEON_ERR_NO_KEY, "no key for Galois element %llu", galois);
    cudaStreamSynchronize(ctx->stream); // the key may be in use by queued work
    ctx->keys.erase(it);
    return FHEON_OK;
}

int fheon_key_stats(const fheon_ctx *ctx, uint32_t *count, uint64_t *bytes)
{
    if (!ctx) return FHEON_ERR_ARG;
    u64 b = 0;
    for (auto &kv : ctx->keys) b += kv.second.mem.bytes;
    if (count) *count = (u32)ctx->keys.size();
    if (bytes) *bytes = b;
    return FHEON_OK;
}

int fheon_key_download(fheon_ctx *ctx, uint64_t galois, uint64_t *host)
{
    if (!ctx || !host) return FHEON_ERR_ARG;
    auto it = ctx->keys.find(galois);
    if (it == ctx->keys.end()) return fail(ctx, FHEON_ERR_NO_KEY, "no key for Galois element %llu", galois);
    const size_t per = (size_t)(ctx->L + ctx->K);
    DevMem tmp;
    if (!tmp.alloc(it->second.mem.bytes, ctx->stream)) return fail(ctx, FHEON_ERR_OOM, "key download buffer");
    FHEON_CUDA(ctx, key_from_mont(ctx, it->second.mem.as<u64>(), tmp.as<u64>(), per, 2 * ctx->beta));
    return download(ctx, tmp.p, host, it->second.mem.bytes);
}

int fheon_key_upload(fheon_ctx *ctx, uint64_t galois, const uint64_t *host)
{
    if (!ctx || !host) return FHEON_ERR_ARG;
    if (galois != 0 && ((galois & 1) == 0 || galois >= 2ull * ctx->N))
        return fail(ctx, FHEON_ERR_ARG, "bad Galois element %llu", (unsigned long long)galois);
    const size_t per = (size_t)(ctx->L + ctx->K), blocks = (size_t)2 * ctx->beta, N = ctx->N;
    for (size_t b = 0; b < blocks; b++)
        for (size_t t = 0; t < per; t++) {
            const u64 q = ctx->mod[t];
            const uint64_t *x = host + (b * per + t) * N;
            for (size_t i = 0; i < N; i++)
                if (x[i] >= q)
                    return fail(ctx, FHEON_ERR_ARG, "key upload: residue %zu of limb %zu in block %zu is not below its modulus",
                                i, t, b);
        }
    const size_t bytes = blocks * per * N * 8;
    auto it = ctx->keys.find(galois);
    RotKey fresh;
    u64 *dst;
    if (it != ctx->keys.end()) {
        // overwritten where it is, so that captured graphs still read it;
        // queued work may be reading the old values
        FHEON_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        dst = it->second.mem.as<u64>();
    } else {
        if (!fresh.mem.alloc(bytes, ctx->stream)) return fail(ctx, FHEON_ERR_OOM, "key upload (%zu bytes)", bytes);
        dst = fresh.mem.as<u64>();
    }
    FHEON_CUDA(ctx, cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    FHEON_CUDA(ctx, key_to_mont(ctx, dst, per, (u32)blocks));
    FHEON_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (it == ctx->keys.end()) ctx->keys.emplace(galois, std::move(fresh));
    return FHEON_OK;
}

int fheon_key_list(const fheon_ctx *ctx, uint64_t *out, uint32_t *n)
{
    if (!ctx || !n) return FHEON_ERR_ARG;
    const u32 have = (u32)ctx->keys.size();
    if (out) {
        if (*n < have) return FHEON_ERR_ARG;
        u32 i = 0;
        for (auto &kv : ctx->keys) out[i++] = kv.first; // std::map: increasing order
    }
    *n = have;
    return FHEON_OK;
}

// ------------------------------------------------------------------ plaintexts
int fheon_plain_from_coeffs(fheon_ctx *ctx, const int64_t *coeffs, uint32_t level, double scale, fheon_pt **out)
{
    if (!ctx || !coeffs || !out || level < 1 || level > ctx->L) return FHEON_ERR_ARG;
    fheon_pt *pt = new fheon_pt();
    pt->level = level;
    pt->scale = scale;
    int rc = plain_from_coeffs_dev(ctx, coeffs, level, pt);
    if (rc) { delete pt; return rc; }
    *out = pt;
    return FHEON_OK;
}

int fheon_encode_plain(fheon_ctx *ctx, const double *re, const double *im, uint32_t n, uint32_t level,
                       double scale, fheon_pt **out)
{
    if (!ctx || !re || !out || n > ctx->N / 2 || level < 1 || level > ctx->L || !(scale > 0)) return FHEON_ERR_ARG;
    fheon_pt *pt = new fheon_pt();
    pt->level = level;
    pt->scale = scale;
    int rc = encode_dev(ctx, re, im, n, scale, level, pt, nullptr);
    if (rc) { delete pt; return rc; }
    *out = pt;
    return FHEON_OK;
}

int fheon_encode_coeffs(fheon_ctx *ctx, const double *re, const double *im, uint32_t n, double scale,
                        int64_t *coeffs)
{
    if (!ctx || !re || !coeffs || n > ctx->N / 2 || !(scale > 0)) return FHEON_ERR_ARG;
    return encode_dev(ctx, re, im, n, scale, 0, nullptr, coeffs);
}

int fheon_decode(fheon_ctx *ctx, const fheon_pt *pt, double *re, double *im, uint32_t n)
{
    if (!ctx || !pt || !re || n > ctx->N / 2) return FHEON_ERR_ARG;
    return decode_dev(ctx, pt, re, im, n);
}

int fheon_pt_info(const fheon_pt *pt, uint32_t *level, double *scale)
{
    if (!pt) return FHEON_ERR_ARG;
    if (level) *level = pt->level;
    if (scale) *scale = pt->scale;
    return FHEON_OK;
}
int fheon_pt_download(fheon_ctx *ctx, const fheon_pt *pt, uint64_t *host)
{
    if (!ctx || !pt || !host) return FHEON_ERR_ARG;
    return download(ctx, pt->m.p, host, (size_t)pt->level * ctx->limb_bytes());
}
int fheon_pt_destroy(fheon_pt *pt) { delete pt; return FHEON_OK; }

// ------------------------------------------------------------------ ciphertexts
int fheon_encrypt_seeded(fheon_ctx *ctx, const fheon_pk *pk, const fheon_pt *pt, uint64_t nonce, fheon_ct **out)
{
    if (!ctx || !pk || !pt || !out) return FHEON_ERR_ARG;
    if (pt->level != ctx->L) return fail(ctx, FHEON_ERR_LEVEL, "encrypt needs a plaintext at level L");
    fheon_ct *ct = new fheon_ct();
    int rc = encrypt_dev(ctx, pk, pt, nonce, ct);
    if (rc) { delete ct; return rc; }
    ct->scale = pt->scale;
    *out = ct;
    return FHEON_OK;
}
int fheon_encrypt(fheon_ctx *ctx, const fheon_pk *pk, const fheon_pt *pt, fheon_ct **out)
{
    if (!ctx) return FHEON_ERR_ARG;
    return fheon_encrypt_seeded(ctx, pk, pt, (1ull << 63) | ctx->enc_counter++, out);
}

int fheon_decrypt(fheon_ctx *ctx, const fheon_sk *sk, const fheon_ct *ct, fheon_pt **out)
{
    if (!ctx || !sk || !ct || !out) return FHEON_ERR_ARG;
    fheon_pt *pt = new fheon_pt();
    pt->level = ct->level;
    pt->scale = ct->scale;
    if (!pt->m.alloc((size_t)ct->level * ctx->limb_bytes(), ctx->stream)) {
        delete pt;
        return fail(ctx, FHEON_ERR_OOM, "plaintext allocation");
    }
    cudaError_t e = k_decrypt(ctx, ct->c0(), sk->s.as<u64>(), pt->m.as<u64>(), ct->level);
    if (e != cudaSuccess) { delete pt; return cuda_fail(ctx, e, "decrypt"); }
    *out = pt;
    return FHEON_OK;
}

int fheon_ct_create(fheon_ctx *ctx, uint32_t level, double scale, fheon_ct **out)
{
    if (!ctx || !out || level < 1 || level > ctx->L) return FHEON_ERR_ARG;
    fheon_ct *ct = new fheon_ct();
    int rc = ct_reshape(ctx, ct, level);
    if (rc) { delete ct; return rc; }
    ct->scale = scale;
    cudaError_t e = cudaMemsetAsync(ct->c.p, 0, (size_t)2 * level * ctx->limb_bytes(), ctx->stream);
    if (e != cudaSuccess) { delete ct; return cuda_fail(ctx, e, "memset"); }
    *out = ct;
    return FHEON_OK;
}
int fheon_ct_destroy(fheon_ct *ct) { delete ct; return FHEON_OK; }

int fheon_ct_create_batch(fheon_ctx *ctx, const uint32_t *levels, uint32_t n, double scale, fheon_ct **out)
{
    if (!ctx || !levels || !out || !n) return FHEON_ERR_ARG;
    size_t total = 0;
    for (u32 i = 0; i < n; i++) {
        if (levels[i] < 1 || levels[i] > ctx->L) return FHEON_ERR_ARG;
        total += (size_t)2 * levels[i] * ctx->limb_bytes();
    }
    auto block = std::make_shared<DevMem>();
    if (!block->alloc(total, ctx->stream)) return fail(ctx, FHEON_ERR_OOM, "ciphertext batch of %zu bytes", total);
    FHEON_CUDA(ctx, cudaMemsetAsync(block->p, 0, total, ctx->stream));
    char *base = block->as<char>();
    for (u32 i = 0; i < n; i++) {
        const size_t b = (size_t)2 * levels[i] * ctx->limb_bytes();
        fheon_ct *ct = new fheon_ct();
        ct->c.view(base, b);
        ct->block = block;
        ct->level = ct->cap = levels[i];
        ct->scale = scale;
        out[i] = ct;
        base += b;
    }
    return FHEON_OK;
}

// true when cts[0..n) sit back to back in one batch allocation at their created levels
static bool contiguous(const fheon_ct *const *cts, uint32_t n, size_t limb_bytes, size_t *bytes)
{
    const char *next = nullptr;
    size_t total = 0;
    for (u32 i = 0; i < n; i++) {
        const fheon_ct *c = cts[i];
        if (!c || !c->block || c->level != c->cap || c->block != cts[0]->block) return false;
        if (next && (const char *)c->c.p != next) return false;
        const size_t b = (size_t)2 * c->level * limb_bytes;
        next = (const char *)c->c.p + b;
        total += b;
    }
    *bytes = total;
    return true;
}

int fheon_ct_upload_many_async(fheon_ctx *ctx, fheon_ct *const *cts, uint32_t n, const uint64_t *host, void *stream)
{
    if (!ctx || !cts || !host) return FHEON_ERR_ARG;
    const cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    size_t bytes = 0;
    if (n && contiguous(cts, n, ctx->limb_bytes(), &bytes)) {
        FHEON_CUDA(ctx, cudaMemcpyAsync(cts[0]->c.p, host, bytes, cudaMemcpyHostToDevice, st));
        return FHEON_OK;
    }
    for (u32 i = 0; i < n; i++) {
        if (!cts[i]) return FHEON_ERR_ARG;
        const size_t b = (size_t)2 * cts[i]->level * ctx->limb_bytes();
        FHEON_CUDA(ctx, cudaMemcpyAsync(cts[i]->c.p, host, b, cudaMemcpyHostToDevice, st));
        host += b / 8;
    }
    return FHEON_OK;
}

int fheon_ct_download_many_async(fheon_ctx *ctx, const fheon_ct *const *cts, uint32_t n, uint64_t *host, void *stream)
{
    if (!ctx || !cts || !host) return FHEON_ERR_ARG;
    const cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    size_t bytes = 0;
    if (n && contiguous(cts, n, ctx->limb_bytes(), &bytes)) {
        FHEON_CUDA(ctx, cudaMemcpyAsync(host, cts[0]->c.p, bytes, cudaMemcpyDeviceToHost, st));
        return FHEON_OK;
    }
    for (u32 i = 0; i < n; i++) {
        if (!cts[i]) return FHEON_ERR_ARG;
        const size_t b = (size_t)2 * cts[i]->level * ctx->limb_bytes();
        FHEON_CUDA(ctx, cudaMemcpyAsync(host, cts[i]->c.p, b, cudaMemcpyDeviceToHost, st));
        host += b / 8;
    }
    return FHEON_OK;
}
int fheon_ct_info(const fheon_ct *ct, uint32_t *level, double *scale)
{
    if (!ct) return FHEON_ERR_ARG;
    if (level) *level = ct->level;
    if (scale) *scale = ct->scale;
    return FHEON_OK;
}
int fheon_ct_upload(fheon_ctx *ctx, fheon_ct *ct, const uint64_t *host)
{
    if (!ctx || !ct || !host) return FHEON_ERR_ARG;
    FHEON_CUDA(ctx, cudaMemcpyAsync(ct->c.p, host, (size_t)2 * ct->level * ctx->limb_bytes(),
                                    cudaMemcpyHostToDevice, ctx->stream));
    return FHEON_OK;
}
int fheon_ct_upload_async(fheon_ctx *ctx, fheon_ct *ct, const uint64_t *host, void *stream)
{
    if (!ctx || !ct || !host) return FHEON_ERR_ARG;
    FHEON_CUDA(ctx, cudaMemcpyAsync(ct->c.p, host, (size_t)2 * ct->level * ctx->limb_bytes(), cudaMemcpyHostToDevice,
                                    stream ? (cudaStream_t)stream : ctx->stream));
    return FHEON_OK;
}
int fheon_ct_download_async(fheon_ctx *ctx, const fheon_ct *ct, uint64_t *host, void *stream)
{
    if (!ctx || !ct || !host) return FHEON_ERR_ARG;
    FHEON_CUDA(ctx, cudaMemcpyAsync(host, ct->c.p, (size_t)2 * ct->level * ctx->limb_bytes(), cudaMemcpyDeviceToHost,
                                    stream ? (cudaStream_t)stream : ctx->stream));
    return FHEON_OK;
}
int fheon_ct_download(fheon_ctx *ctx, const fheon_ct *ct, uint64_t *host)
{
    if (!ctx || !ct || !host) return FHEON_ERR_ARG;
    return download(ctx, ct->c.p, host, (size_t)2 * ct->level * ctx->limb_bytes());
}
int fheon_ct_device_ptr(const fheon_ct *ct, void **dptr)
{
    if (!ct || !dptr) return FHEON_ERR_ARG;
    *dptr = ct->c.p;
    return FHEON_OK;
}

// ------------------------------------------------------------------ evaluation
int fheon_rotate_galois(fheon_ctx *ctx, const fheon_ct *in, uint64_t galois, fheon_ct *out)
{
    if (!ctx || !in || !out) return FHEON_ERR_ARG;
    if ((galois & 1) == 0 || galois >= 2ull * ctx->N) return fail(ctx, FHEON_ERR_ARG, "bad Galois element");
    return rotate_one(ctx, in, galois, out);
}
int fheon_rotate(fheon_ctx *ctx, const fheon_ct *in, int32_t step, fheon_ct *out)
{
    if (!ctx) return FHEON_ERR_ARG;
    return fheon_rotate_galois(ctx, in, fheon_galois_elt(ctx, step), out);
}
int fheon_rotate_batch(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n)
{
    if (!ctx || (n && !items)) return FHEON_ERR_ARG;
    return rotate_many(ctx, items, n);
}
int fheon_rotate_hoisted(fheon_ctx *ctx, const fheon_ct *in, const int32_t *steps, uint32_t n, fheon_ct *const *outs)
{
    if (!ctx || !in || (n && (!steps || !outs))) return FHEON_ERR_ARG;
    return rotate_hoisted(ctx, in, steps, n, outs);
}
int fheon_rotate_batch_hoisted(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n)
{
    if (!ctx || (n && !items)) return FHEON_ERR_ARG;
    return rotate_many(ctx, items, n, true);
}

static bool scales_match(double a, double b) { return std::fabs(a - b) <= 1e-9 * std::fabs(a); }

int fheon_mul_plain(fheon_ctx *ctx, const fheon_ct *ct, const fheon_pt *pt, fheon_ct *out)
{
    if (!ctx || !ct || !pt || !out) return FHEON_ERR_ARG;
    if (pt->level < ct->level) return fail(ctx, FHEON_ERR_LEVEL, "plaintext level %u < ciphertext level %u", pt->level, ct->level);
    const u32 l = ct->level;
    const double sc = ct->scale * pt->scale;
    if (out != ct) {
        int rc = ct_reshape(ctx, out, l);
        if (rc) return rc;
    }
    FHEON_CUDA(ctx, k_mul_plain(ctx, ct->c0(), pt->m.as<u64>(), out->c0(), l, 0));
    out->scale = sc;
    return FHEON_OK;
}

int fheon_mac_plain(fheon_ctx *ctx, const fheon_ct *const *cts, const fheon_pt *const *pts, uint32_t n, fheon_ct *out)
{
    if (!ctx || !cts || !pts || !out || n == 0) return FHEON_ERR_ARG;
    for (u32 t = 0; t < n; t++)
        if (!cts[t] || !pts[t]) return fail(ctx, FHEON_ERR_ARG, "mac_plain: null operand %u", t);
    const u32 l = cts[0]->level;
    const double sc = cts[0]->scale * pts[0]->scale;
    std::vector<const u64 *> cp(n), pp(n);
    for (u32 t = 0; t < n; t++) {
        if (cts[t]->level != l) return fail(ctx, FHEON_ERR_LEVEL, "mac_plain: ciphertext %u at level %u, not %u", t, cts[t]->level, l);
        if (pts[t]->level < l) return fail(ctx, FHEON_ERR_LEVEL, "mac_plain: plaintext %u below level %u", t, l);
        if (!scales_match(cts[t]->scale * pts[t]->scale, sc)) return fail(ctx, FHEON_ERR_SCALE, "mac_plain: product %u scale differs", t);
        if (cts[t] == out) return fail(ctx, FHEON_ERR_ARG, "mac_plain: output aliases input %u", t);
        cp[t] = cts[t]->c0();
        pp[t] = pts[t]->m.as<u64>();
    }
    int rc = ct_reshape(ctx, out, l);
    if (rc) return rc;
    FHEON_CUDA(ctx, k_mac_plain(ctx, cp.data(), pp.data(), n, out->c0(), l));
    out->scale = sc;
    return FHEON_OK;
}

int fheon_add(fheon_ctx *ctx, const fheon_ct *a, const fheon_ct *b, fheon_ct *out)
{
    if (!ctx || !a || !b || !out) return FHEON_ERR_ARG;
    if (a->level != b->level) return fail(ctx, FHEON_ERR_LEVEL, "add: levels %u and %u", a->level, b->level);
    if (!scales_match(a->scale, b->scale)) return fail(ctx, FHEON_ERR_SCALE, "add: scales differ");
    const u32 l = a->level;
    const double sc = a->scale;
    if (out != a && out != b) {
        int rc = ct_reshape(ctx, out, l);
        if (rc) return rc;
    }
    FHEON_CUDA(ctx, k_add(ctx, a->c0(), b->c0(), out->c0(), l, 2));
    out->scale = sc;
    return FHEON_OK;
}

int fheon_add_plain(fheon_ctx *ctx, const fheon_ct *ct, const fheon_pt *pt, fheon_ct *out)
{
    if (!ctx || !ct || !pt || !out) return FHEON_ERR_ARG;
    if (pt->level < ct->level) return fail(ctx, FHEON_ERR_LEVEL, "add_plain: plaintext level too low");
    if (!scales_match(ct->scale, pt->scale)) return fail(ctx, FHEON_ERR_SCALE, "add_plain: scales differ");
    const u32 l = ct->level;
    const double sc = ct->scale;
    if (out != ct) {
        int rc = ct_reshape(ctx, out, l);
        if (rc) return rc;
    }
    FHEON_CUDA(ctx, k_add_plain(ctx, ct->c0(), pt->m.as<u64>(), out->c0(), l));
    out->scale = sc;
    return FHEON_OK;
}

} // extern "C"

namespace fheon {
int mul_relin_at(fheon_ctx *ctx, const fheon_ct *a, const fheon_ct *b, u32 l, bool twice, fheon_ct *out)
{
    auto it = ctx->keys.find(0);
    if (it == ctx->keys.end()) return fail(ctx, FHEON_ERR_NO_KEY, "no relinearisation key");
    if (l < 1 || l > a->level || l > b->level) return fail(ctx, FHEON_ERR_LEVEL, "mul_relin: level %u", l);
    const u32 N = ctx->N;
    const double sc = a->scale * b->scale;
    int rc = ensure_workspace(ctx, ctx->ks_ws_limbs(ctx->L) + 3 * (size_t)ctx->L);
    if (rc) return rc;
    u64 *ws = ctx->ws.as<u64>();
    u64 *d = ws + ctx->ks_ws_limbs(ctx->L) * N; // tensor [3][l][N] past the key-switching workspace
    FHEON_CUDA(ctx, k_tensor(ctx, a->c0(), a->c1(N), b->c0(), b->c1(N), d, l, twice));
    if ((rc = ct_reshape(ctx, out, l))) return rc;
    // key-switch d2 from s^2 to s (g = 1: no automorphism); d0 joins component 0, d1 component 1
    if ((rc = keyswitch_rotate(ctx, d, d + (size_t)2 * l * N, l, 1, it->second.mem.as<u64>(), ws, out->c0(),
                               d + (size_t)l * N)))
        return rc;
    out->scale = sc;
    return FHEON_OK;
}

} // namespace fheon

extern "C" {

int fheon_mul_relin(fheon_ctx *ctx, const fheon_ct *a, const fheon_ct *b, fheon_ct *out)
{
    if (!ctx || !a || !b || !out) return FHEON_ERR_ARG;
    if (a->level != b->level) return fail(ctx, FHEON_ERR_LEVEL, "mul_relin: levels %u and %u", a->level, b->level);
    return mul_relin_at(ctx, a, b, a->level, false, out);
}

int fheon_mul_int(fheon_ctx *ctx, const fheon_ct *ct, int64_t v, fheon_ct *out)
{
    if (!ctx || !ct || !out) return FHEON_ERR_ARG;
    const u32 l = ct->level;
    const double sc = ct->scale;
    int rc = out == ct ? FHEON_OK : ct_reshape(ctx, out, l);
    if (rc) return rc;
    FHEON_CUDA(ctx, k_mul_int(ctx, ct->c0(), v, out->c0(), l, 2));
    out->scale = sc;
    return FHEON_OK;
}

int fheon_add_int(fheon_ctx *ctx, const fheon_ct *ct, int64_t v, fheon_ct *out)
{
    if (!ctx || !ct || !out) return FHEON_ERR_ARG;
    const u32 l = ct->level;
    const double sc = ct->scale;
    int rc = out == ct ? FHEON_OK : ct_reshape(ctx, out, l);
    if (rc) return rc;
    FHEON_CUDA(ctx, k_add_int(ctx, ct->c0(), v, out->c0(), l));
    out->scale = sc;
    return FHEON_OK;
}

} // extern "C"

// llround(x) when it fits comfortably in 63 bits
bool fheon::round_int(double x, int64_t *v)
{
    if (!std::isfinite(x) || std::fabs(x) >= 4611686018427387904.0) return false; // 2^62
    *v = (int64_t)std::llround(x);
    return true;
}

extern "C" {

int fheon_add_const(fheon_ctx *ctx, const fheon_ct *ct, double c, fheon_ct *out)
{
    if (!ctx || !ct || !out) return FHEON_ERR_ARG;
    int64_t v;
    if (!round_int(c * ct->scale, &v)) return fail(ctx, FHEON_ERR_ARG, "add_const: c * scale out of range");
    return fheon_add_int(ctx, ct, v, out);
}

int fheon_mul_const_rescale(fheon_ctx *ctx, const fheon_ct *ct, double c, double target, fheon_ct *out)
{
    if (!ctx || !ct || !out || !(target > 0)) return FHEON_ERR_ARG;
    return mul_const_rescale_at(ctx, ct, ct->level, c, target, out);
}

} // extern "C"

int fheon::mul_const_rescale_at(fheon_ctx *ctx, const fheon_ct *ct, u32 l, double c, double target, fheon_ct *out)
{
    if (l < 2 || l > ct->level) return fail(ctx, FHEON_ERR_LEVEL, "mul_const_rescale needs 2 <= level <= %u", ct->level);
    int64_t K;
    if (!round_int(((c * target) * (double)ctx->mod[l - 1]) / ct->scale, &K))
        return fail(ctx, FHEON_ERR_ARG, "mul_const_rescale: constant factor out of range");
    const double sc = ct->scale;
    const u64 stride = (u64)ct->level * ctx->N;
    const u64 *src = ct->c0();
    int rc;
    if (out == ct) {
        if (l != ct->level) return fail(ctx, FHEON_ERR_ARG, "mul_const_rescale: in place needs the full level");
    } else if ((rc = ct_reshape(ctx, out, l))) {
        return rc;
    }
    FHEON_CUDA(ctx, k_mul_int(ctx, src, K, out->c0(), l, 2, stride));
    out->scale = sc;
    if ((rc = rescale_ct(ctx, out, out))) return rc;
    out->scale = target;
    return FHEON_OK;
}

extern "C" {

int fheon_rescale(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !in || !out) return FHEON_ERR_ARG;
    if (in->level < 2) return fail(ctx, FHEON_ERR_LEVEL, "rescale needs level >= 2");
    return rescale_ct(ctx, in, out);
}

int fheon_drop_level(fheon_ctx *ctx, const fheon_ct *in, uint32_t level, fheon_ct *out)
{
    if (!ctx || !in || !out || level < 1 || level > in->level) return FHEON_ERR_ARG;
    const size_t lb = ctx->limb_bytes();
    if (out == in) {
        // move c1's lowest limbs down next to c0's, one limb at a time so that
        // no copy overlaps itself and no source limb is overwritten first
        u64 *c1 = in->c1(ctx->N);
        for (u32 i = 0; i < level && level < in->level; i++)
            FHEON_CUDA(ctx, cudaMemcpyAsync(in->c0() + (size_t)(level + i) * ctx->N, c1 + (size_t)i * ctx->N, lb,
                                            cudaMemcpyDeviceToDevice, ctx->stream));
        out->level = level;
        return FHEON_OK;
    }
    int rc = ct_reshape(ctx, out, level);
    if (rc) return rc;
    FHEON_CUDA(ctx, cudaMemcpyAsync(out->c0(), in->c0(), level * lb, cudaMemcpyDeviceToDevice, ctx->stream));
    FHEON_CUDA(ctx, cudaMemcpyAsync(out->c1(ctx->N), in->c1(ctx->N), level * lb, cudaMemcpyDeviceToDevice, ctx->stream));
    out->scale = in->scale;
    return FHEON_OK;
}

} // extern "C"
