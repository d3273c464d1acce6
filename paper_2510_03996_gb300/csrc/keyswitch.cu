// keyswitch.cu -- the homomorphic rotation: Galois automorphism + hybrid key
// switching (paper Sec. 2.2 rotation, Sec. 6 "4 digits"; Han-Ki hybrid key
// switching with Cheon et al. fast base conversion).
//
// Pipeline for one ciphertext (c0, c1) at level l, Galois element g,
// beta = ceil(l/alpha) digits, all in the evaluation domain:
//   1  INTT of sigma_g(c1)   -- the automorphism is a gather in the first
//                               pass's load; the last pass multiplies by
//                               N^-1 * Dhat_i^-1, giving the ModUp inputs
//   2  ModUp base conversion -- digit j's limbs to every other limb of Q_l u P
//   3  NTT of the new limbs  -- beta*(l+K) - l transforms
//   4  key inner product     -- acc_b[t] = sum_j d_j[t] * key_g[j][b][t];
//                               digit limbs come straight from sigma_g(c1)
//   5  INTT of acc's P limbs -- times N^-1 * Phat_k^-1
//   6  ModDown conversion    -- P -> each q_i
//   7  NTT of the converted limbs
//   8  out_b = (acc_b - conv_b) * P^-1 (+ sigma_g(c0) for b = 0)
// Workspace per ciphertext (limbs of N u64): xt[l] | ext[beta][l+K] |
// acc[2][l+K] | pc[2][K] | conv[2][l].
#include "jobs.cuh"

namespace fheon {

namespace {

constexpr int TPB = 256;

// Step 2.  One thread per coefficient n, blockIdx.y = digit j.
__global__ void __launch_bounds__(TPB) modup_bconv_kernel(const u64 *__restrict__ xt, u64 *__restrict__ ext, u32 level,
                                                          u32 K, u32 L, u32 alpha, u32 N,
                                                          const u64 *__restrict__ conv_tab,
                                                          const ModConst *__restrict__ mc)
{
    const u32 n = blockIdx.x * TPB + threadIdx.x;
    const u32 j = blockIdx.y;
    if (n >= N) return;
    const u32 d0 = j * alpha, d = min(alpha, level - d0), nl = level + K, nm = L + K;
    u64 x[16];
#pragma unroll
    for (u32 i = 0; i < 16; i++)
        if (i < d) x[i] = xt[(u64)(d0 + i) * N + n];
    const u64 *tab = conv_tab + ((u64)j * alpha + (d - 1)) * alpha * nm;
    u64 *o = ext + (u64)j * nl * N + n;
    for (u32 t = 0; t < nl; t++) {
        if (t >= d0 && t < d0 + d) continue;
        const u32 m = limb_modidx(t, level, L);
        u128acc a;
        acc_zero(a);
#pragma unroll
        for (u32 i = 0; i < 16; i++)
            if (i < d) acc_mad(a, x[i], __ldg(&tab[i * nm + m]));
        const ModConst c = mc[m];
        o[(u64)t * N] = redc_acc(a, c.q, c.qneg_inv);
    }
}

// Step 4.  Two coefficients per thread; blockIdx.y = limb t of Q_l u P.
__global__ void __launch_bounds__(TPB) ks_inner_kernel(const u64 *__restrict__ c1, u64 g, const u64 *__restrict__ ext,
                                                       const u64 *__restrict__ key, u64 *__restrict__ acc, u32 level,
                                                       u32 K, u32 L, u32 alpha, u32 N, u32 logN,
                                                       const ModConst *__restrict__ mc)
{
    const u32 n = (blockIdx.x * TPB + threadIdx.x) * 2;
    if (n >= N) return;
    const u32 t = blockIdx.y, nl = level + K, nm = L + K;
    const u32 m = limb_modidx(t, level, L);
    const u32 beta = (level + alpha - 1) / alpha;
    u128acc a0x, a0y, a1x, a1y;
    acc_zero(a0x); acc_zero(a0y); acc_zero(a1x); acc_zero(a1y);
    for (u32 j = 0; j < beta; j++) {
        ulonglong2 dv;
        if (t < level && t / alpha == j) {
            const u64 *src = c1 + (u64)t * N;
            dv.x = src[automorph_src(n, g, logN)];
            dv.y = src[automorph_src(n + 1, g, logN)];
        } else {
            dv = *reinterpret_cast<const ulonglong2 *>(ext + ((u64)j * nl + t) * N + n);
        }
        const ulonglong2 kb = __ldg(reinterpret_cast<const ulonglong2 *>(key + (((u64)j * 2 + 0) * nm + m) * N + n));
        const ulonglong2 ka = __ldg(reinterpret_cast<const ulonglong2 *>(key + (((u64)j * 2 + 1) * nm + m) * N + n));
        acc_mad(a0x, dv.x, kb.x);
        acc_mad(a0y, dv.y, kb.y);
        acc_mad(a1x, dv.x, ka.x);
        acc_mad(a1y, dv.y, ka.y);
    }
    const ModConst c = mc[m];
    *reinterpret_cast<ulonglong2 *>(acc + ((u64)0 * nl + t) * N + n) =
        make_ulonglong2(redc_acc(a0x, c.q, c.qneg_inv), redc_acc(a0y, c.q, c.qneg_inv));
    *reinterpret_cast<ulonglong2 *>(acc + ((u64)1 * nl + t) * N + n) =
        make_ulonglong2(redc_acc(a1x, c.q, c.qneg_inv), redc_acc(a1y, c.q, c.qneg_inv));
}

// Step 6.  One thread per coefficient; blockIdx.y = component b.
__global__ void __launch_bounds__(TPB) moddown_bconv_kernel(const u64 *__restrict__ pc, u64 *__restrict__ conv,
                                                            u32 level, u32 K, u32 L, u32 N,
                                                            const u64 *__restrict__ conv_tab,
                                                            const ModConst *__restrict__ mc)
{
    const u32 n = blockIdx.x * TPB + threadIdx.x;
    if (n >= N) return;
    const u32 b = blockIdx.y;
    u64 x[16];
#pragma unroll
    for (u32 k = 0; k < 16; k++)
        if (k < K) x[k] = pc[((u64)b * K + k) * N + n];
    for (u32 i = 0; i < level; i++) {
        u128acc a;
        acc_zero(a);
#pragma unroll
        for (u32 k = 0; k < 16; k++)
            if (k < K) acc_mad(a, x[k], __ldg(&conv_tab[(u64)k * L + i]));
        const ModConst c = mc[i];
        conv[((u64)b * level + i) * N + n] = redc_acc(a, c.q, c.qneg_inv);
    }
}

// Step 8.  out[b][i][n] = (acc[b][i][n] - conv[b][i][n]) * P^-1 (+ c0[i][src(n)] when b = 0).
__global__ void __launch_bounds__(TPB) moddown_combine_kernel(const u64 *__restrict__ acc,
                                                              const u64 *__restrict__ conv,
                                                              const u64 *__restrict__ c0, u64 g,
                                                              u64 *__restrict__ out, u32 level, u32 K, u32 N,
                                                              u32 logN, const ulonglong2 *__restrict__ pinv,
                                                              const ModConst *__restrict__ mc)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    const u64 per = (u64)level * N;
    if (idx >= 2 * per) return;
    const u32 b = (u32)(idx / per);
    const u32 i = (u32)((idx % per) / N), n = (u32)(idx % N);
    const u64 q = mc[i].q;
    const u64 a = acc[((u64)b * (level + K) + i) * N + n];
    const u64 v = conv[((u64)b * level + i) * N + n];
    const ulonglong2 pi = pinv[i];
    u64 r = shoup(a + q - v, pi.x, pi.y, q);
    if (b == 0) r = addmod(r, c0[(u64)i * N + automorph_src(n, g, logN)], q);
    out[idx] = r;
}

} // namespace

// Run the whole pipeline for one ciphertext.  `ws` holds ks_ws_limbs(l) limbs.
int keyswitch_rotate(fheon_ctx *ctx, const u64 *c0, const u64 *c1, u32 l, u64 g, const u64 *key, u64 *ws, u64 *out)
{
    const u32 N = ctx->N, K = ctx->K, L = ctx->L, A = ctx->alpha, beta = ctx->beta_at(l);
    cudaStream_t st = ctx->stream;
    u64 *xt = ws;
    u64 *ext = xt + (u64)l * N;
    u64 *acc = ext + (u64)beta * (l + K) * N;
    u64 *pc = acc + (u64)2 * (l + K) * N;
    u64 *conv = pc + (u64)2 * K * N;
    const ModConst *mc = ctx->tab.mc.as<ModConst>();

    // 1: INTT(sigma_g(c1)) scaled for ModUp
    {
        MapParams mp = map_params(ctx, c1, xt, l, 0, l);
        mp.gather_g = g;
        mp.scale_mode = SCALE_MODUP;
        mp.scale_tab = ctx->tab.modup_scale.as<ulonglong2>();
        FHEON_CUDA(ctx, (ntt::launch<true, MapJob>(ctx->logN, mp, l, st)));
    }
    // 2: ModUp base conversion
    modup_bconv_kernel<<<dim3((N + TPB - 1) / TPB, beta), TPB, 0, st>>>(xt, ext, l, K, L, A, N,
                                                                         ctx->tab.modup_conv.as<u64>(), mc);
    prof_mark(st, "modup_bconv");
    FHEON_CUDA(ctx, cudaGetLastError());
    // 3: NTT of the converted limbs (digit limbs skipped)
    {
        MapParams mp = map_params(ctx, ext, ext, l + K, 0, l);
        mp.skip_digit = 1;
        FHEON_CUDA(ctx, (ntt::launch<false, MapJob>(ctx->logN, mp, beta * (l + K), st)));
    }
    // 4: inner product with the key
    ks_inner_kernel<<<dim3((N / 2 + TPB - 1) / TPB, l + K), TPB, 0, st>>>(c1, g, ext, key, acc, l, K, L, A, N,
                                                                          ctx->logN, mc);
    prof_mark(st, "ks_inner");
    FHEON_CUDA(ctx, cudaGetLastError());
    // 5: INTT of the P limbs of both components
    {
        MapParams mp = map_params(ctx, acc + (u64)l * N, pc, K, l, l);
        mp.in_poly_stride = (u64)(l + K) * N;
        mp.out_poly_stride = (u64)K * N;
        mp.scale_mode = SCALE_MODDOWN;
        mp.scale_tab = ctx->tab.moddown_scale.as<ulonglong2>();
        FHEON_CUDA(ctx, (ntt::launch<true, MapJob>(ctx->logN, mp, 2 * K, st)));
    }
    // 6: ModDown base conversion P -> Q_l
    moddown_bconv_kernel<<<dim3((N + TPB - 1) / TPB, 2), TPB, 0, st>>>(pc, conv, l, K, L, N,
                                                                       ctx->tab.moddown_conv.as<u64>(), mc);
    prof_mark(st, "moddown_bconv");
    FHEON_CUDA(ctx, cudaGetLastError());
    // 7: NTT of the converted limbs
    {
        MapParams mp = map_params(ctx, conv, conv, l, 0, l);
        FHEON_CUDA(ctx, (ntt::launch<false, MapJob>(ctx->logN, mp, 2 * l, st)));
    }
    // 8: combine
    {
        const u64 tot = (u64)2 * l * N;
        moddown_combine_kernel<<<(unsigned)((tot + TPB - 1) / TPB), TPB, 0, st>>>(
            acc, conv, c0, g, out, l, K, N, ctx->logN, ctx->tab.pinv.as<ulonglong2>(), mc);
        prof_mark(st, "moddown_combine");
        FHEON_CUDA(ctx, cudaGetLastError());
    }
    return FHEON_OK;
}

int rotate_one(fheon_ctx *ctx, const fheon_ct *in, u64 g, fheon_ct *out)
{
    auto it = ctx->keys.find(g);
    if (it == ctx->keys.end()) return fail(ctx, FHEON_ERR_NO_KEY, "no rotation key for Galois element %llu", g);
    const u32 l = in->level;
    const size_t need = ctx->ks_ws_limbs(ctx->L) + 2 * (size_t)ctx->L; // + in-place staging
    int rc = ensure_workspace(ctx, need);
    if (rc) return rc;
    u64 *ws = ctx->ws.as<u64>();
    const u64 *c0 = in->c0(), *c1 = in->c1(ctx->N);
    const double sc = in->scale;
    if (out == in) {
        u64 *stage = ws + ctx->ks_ws_limbs(ctx->L) * ctx->N;
        rc = keyswitch_rotate(ctx, c0, c1, l, g, it->second.mem.as<u64>(), ws, stage);
        if (rc) return rc;
        FHEON_CUDA(ctx, cudaMemcpyAsync(out->c0(), stage, (size_t)2 * l * ctx->limb_bytes(),
                                        cudaMemcpyDeviceToDevice, ctx->stream));
        return FHEON_OK;
    }
    rc = ct_reshape(ctx, out, l);
    if (rc) return rc;
    out->scale = sc;
    return keyswitch_rotate(ctx, c0, c1, l, g, it->second.mem.as<u64>(), ws, out->c0());
}

int rotate_many(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n)
{
    for (u32 i = 0; i < n; i++) {
        if (!items[i].in || !items[i].out) return fail(ctx, FHEON_ERR_ARG, "null ciphertext in batch item %u", i);
        int rc = fheon_rotate(ctx, items[i].in, items[i].step, items[i].out);
        if (rc) return rc;
    }
    return FHEON_OK;
}

} // namespace fheon
