// sampler.cu -- every random draw of the scheme, on the device, and the key
// generation / encryption built on them (paper Sec. 5.7: context, keys and the
// encryption layer).
//
// Draws.  Stream (seed, domain, idx) is the ChaCha20 block function (RFC 8439
// Sec. 2.3) with key words (seed lo, seed hi, 0, .., 0), nonce words
// (domain, idx lo, idx hi) and the block counter; 64-bit draw n is the
// little-endian word pair 2(n%8), 2(n%8)+1 of block n/8.  From draws:
//   ternary  : draw mod 3, minus 1
//   Gaussian : smallest k in [-20, 20) with draw < T[k+20], else 20; T is the
//              cumulative table of exp(-k^2 / (2 * 3.2^2)) scaled to 2^64
//   uniform  : (draw 2n+1 * 2^64 + draw 2n) mod q, per limb (its own stream)
// Domains: 1 secret, 2 public a, 3 public e, 4 key-switching a, 5 key-switching
// e, 6 encryption v, 7 encryption e0, 8 encryption e1.
#include <vector>

#include "jobs.cuh"

namespace fheon {

namespace {
constexpr int TPB = 256;
enum : u32 { DOM_SK = 1, DOM_PK_A = 2, DOM_PK_E = 3, DOM_KSK_A = 4, DOM_KSK_E = 5,
             DOM_ENC_V = 6, DOM_ENC_E0 = 7, DOM_ENC_E1 = 8 };

__device__ __forceinline__ u32 rotl(u32 v, int c) { return (v << c) | (v >> (32 - c)); }
#define QR(a, b, c, d)                 \
    a += b; d ^= a; d = rotl(d, 16);   \
    c += d; b ^= c; b = rotl(b, 12);   \
    a += b; d ^= a; d = rotl(d, 8);    \
    c += d; b ^= c; b = rotl(b, 7);

__device__ void chacha_block(u64 seed, u32 domain, u64 idx, u32 counter, u32 out[16])
{
    const u32 s0 = 0x61707865u, s1 = 0x3320646eu, s2 = 0x79622d32u, s3 = 0x6b206574u;
    const u32 k0 = (u32)seed, k1 = (u32)(seed >> 32);
    const u32 n0 = domain, n1 = (u32)idx, n2 = (u32)(idx >> 32);
    u32 x0 = s0, x1 = s1, x2 = s2, x3 = s3, x4 = k0, x5 = k1, x6 = 0, x7 = 0;
    u32 x8 = 0, x9 = 0, x10 = 0, x11 = 0, x12 = counter, x13 = n0, x14 = n1, x15 = n2;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        QR(x0, x4, x8, x12) QR(x1, x5, x9, x13) QR(x2, x6, x10, x14) QR(x3, x7, x11, x15)
        QR(x0, x5, x10, x15) QR(x1, x6, x11, x12) QR(x2, x7, x8, x13) QR(x3, x4, x9, x14)
    }
    out[0] = x0 + s0; out[1] = x1 + s1; out[2] = x2 + s2; out[3] = x3 + s3;
    out[4] = x4 + k0; out[5] = x5 + k1; out[6] = x6; out[7] = x7;
    out[8] = x8; out[9] = x9; out[10] = x10; out[11] = x11;
    out[12] = x12 + counter; out[13] = x13 + n0; out[14] = x14 + n1; out[15] = x15 + n2;
}
#undef QR

__device__ __forceinline__ u64 residue_of_small(long long v, u64 q) { return v >= 0 ? (u64)v : q - (u64)(-v); }

// Small signed samples (ternary / Gaussian) of one stream, as residues in
// `nlimb` limbs: limb position p has modulus index mods[p].  One thread per
// ChaCha block (8 coefficients).  grid.y selects among `nstreams` streams
// with idx = idx0 + y * idx_step and output out + y * out_stride.
template <bool GAUSS>
__global__ void __launch_bounds__(TPB) small_kernel(u64 seed, u32 domain, u64 idx0, u64 idx_step, u64 *out,
                                                    u64 out_stride, u32 N, const u32 *__restrict__ mods, u32 nlimb,
                                                    const u64 *__restrict__ cdt, const ModConst *__restrict__ mc)
{
    __shared__ u64 T[41];
    if (GAUSS && threadIdx.x < 41) T[threadIdx.x] = cdt[threadIdx.x];
    if (GAUSS) __syncthreads();
    const u32 blk = blockIdx.x * TPB + threadIdx.x;
    if (blk * 8 >= N) return;
    u32 w[16];
    chacha_block(seed, domain, idx0 + blockIdx.y * idx_step, blk, w);
    long long v[8];
#pragma unroll
    for (int p = 0; p < 8; p++) {
        const u64 d = (u64)w[2 * p] | ((u64)w[2 * p + 1] << 32);
        if (GAUSS) {
            int k = 0;
            while (k < 40 && d >= T[k]) k++;
            v[p] = k - 20;
        } else {
            v[p] = (long long)(d % 3) - 1;
        }
    }
    u64 *o = out + blockIdx.y * out_stride;
    for (u32 l = 0; l < nlimb; l++) {
        const u64 q = mc[mods[l]].q;
#pragma unroll
        for (int p = 0; p < 8; p++) o[(u64)l * N + blk * 8 + p] = residue_of_small(v[p], q);
    }
}

// Uniform residues: limb position p (modulus mods[p]) of stream y draws from
// stream (seed, domain, idx0 + y*idx_step + p*idx_limb).  One thread per block
// (4 coefficients); grid.z = limb position, grid.y = stream.
__global__ void __launch_bounds__(TPB) uniform_kernel(u64 seed, u32 domain, u64 idx0, u64 idx_step, u64 idx_limb,
                                                      u64 *out, u64 out_stride, u32 N, const u32 *__restrict__ mods,
                                                      const ModConst *__restrict__ mc)
{
    const u32 blk = blockIdx.x * TPB + threadIdx.x;
    if (blk * 4 >= N) return;
    const u32 p = blockIdx.z;
    u32 w[16];
    chacha_block(seed, domain, idx0 + blockIdx.y * idx_step + p * idx_limb, blk, w);
    const ModConst m = mc[mods[p]];
    u64 *o = out + blockIdx.y * out_stride + (u64)p * N + blk * 4;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const u64 lo = (u64)w[4 * c] | ((u64)w[4 * c + 1] << 32);
        const u64 hi = (u64)w[4 * c + 2] | ((u64)w[4 * c + 3] << 32);
        // hi*2^64 + lo = (hi mod q)*2^64 + lo (mod q); the right side is < q*2^64,
        // so REDC followed by a multiply by 2^64 mod q gives the residue exactly.
        const u64 h = redc(__umul64hi(hi, m.r1), hi * m.r1, m.q, m.qneg_inv);
        const u64 r = redc_lazy(h, lo, m.q, m.qneg_inv);
        o[c] = shoup(r, m.r1, m.r1_sh, m.q);
    }
}

// b[t] = -a[t]*s[t] + e[t] (+ P*sfrom[t] when t is in digit `j`; j < 0: never);
// then optionally both b and a to Montgomery form.  Over `nlimb` limbs whose
// modulus index is the limb position.
__global__ void __launch_bounds__(TPB) key_combine_kernel(u64 *b, u64 *a, const u64 *__restrict__ s,
                                                          const u64 *__restrict__ sfrom, u32 nlimb, u32 logN, int j,
                                                          u32 alpha, u32 L, const ulonglong2 *__restrict__ pmod,
                                                          const ModConst *__restrict__ mc, int to_mont_form)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    if (idx >= ((u64)nlimb << logN)) return;
    const u32 t = (u32)(idx >> logN);
    const ModConst m = mc[t];
    const u64 av = a[idx];
    u64 r = submod(b[idx], mulmod_plain(av, s[idx], m), m.q);
    if (j >= 0 && t < L && t / alpha == (u32)j) {
        const ulonglong2 P = pmod[t];
        r = addmod(r, shoup(sfrom[idx], P.x, P.y, m.q), m.q);
    }
    if (to_mont_form) {
        b[idx] = to_mont(r, m);
        a[idx] = to_mont(av, m);
    } else {
        b[idx] = r;
    }
}

// out = in * 2^-64 (Montgomery form back to residues), over blocks of
// `per` limbs whose modulus index is the position within the block.
__global__ void __launch_bounds__(TPB) from_mont_kernel(const u64 *__restrict__ in, u64 *__restrict__ out, u32 per,
                                                        u64 total, u32 logN, const ModConst *__restrict__ mc)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    if (idx >= total) return;
    const ModConst m = mc[(u32)((idx >> logN) % per)];
    out[idx] = redc(0, in[idx], m.q, m.qneg_inv);
}

// x = x * 2^64 mod q in place (residues to Montgomery form), over blocks of
// `per` limbs whose modulus index is the position within the block
__global__ void __launch_bounds__(TPB) to_mont_kernel(u64 *x, u32 per, u64 total, u32 logN,
                                                      const ModConst *__restrict__ mc)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    if (idx >= total) return;
    const ModConst m = mc[(u32)((idx >> logN) % per)];
    x[idx] = to_mont(x[idx], m);
}

// sigma_g gather of an evaluation-form polynomial over `nlimb` limbs
__global__ void __launch_bounds__(TPB) gather_kernel(const u64 *__restrict__ in, u64 *__restrict__ out, u64 g,
                                                     u32 nlimb, u32 logN)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    if (idx >= ((u64)nlimb << logN)) return;
    const u64 base = idx & ~(((u64)1 << logN) - 1);
    out[idx] = in[base + automorph_src((u32)(idx & ((1u << logN) - 1)), g, logN)];
}

// s^2 (pointwise in the evaluation domain) over `nlimb` limbs
__global__ void __launch_bounds__(TPB) square_kernel(const u64 *__restrict__ in, u64 *__restrict__ out, u32 nlimb,
                                                     u32 logN, const ModConst *__restrict__ mc)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    if (idx >= ((u64)nlimb << logN)) return;
    const ModConst m = mc[idx >> logN];
    out[idx] = mulmod_plain(in[idx], in[idx], m);
}

// ct0 = v*pb + e0 + m, ct1 = v*pa + e1 over L limbs
__global__ void __launch_bounds__(TPB) encrypt_combine_kernel(const u64 *__restrict__ v, const u64 *__restrict__ e0,
                                                              const u64 *__restrict__ e1, const u64 *__restrict__ pk,
                                                              const u64 *__restrict__ msg, u64 *__restrict__ ct,
                                                              u32 L, u32 logN, const ModConst *__restrict__ mc)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    const u64 per = (u64)L << logN;
    if (idx >= per) return;
    const ModConst m = mc[(u32)(idx >> logN)];
    const u64 vv = v[idx];
    ct[idx] = addmod(addmod(mulmod_plain(vv, pk[idx], m), e0[idx], m.q), msg[idx], m.q);
    ct[per + idx] = addmod(mulmod_plain(vv, pk[per + idx], m), e1[idx], m.q);
}

// signed 64-bit coefficients -> residues in limbs 0..level-1
__global__ void __launch_bounds__(TPB) coeffs_to_limbs_kernel(const long long *__restrict__ c, u64 *__restrict__ out,
                                                              u32 level, u32 logN, const ModConst *__restrict__ mc)
{
    const u64 idx = (u64)blockIdx.x * TPB + threadIdx.x;
    if (idx >= ((u64)level << logN)) return;
    const ModConst m = mc[(u32)(idx >> logN)];
    const long long v = c[idx & ((1u << logN) - 1)];
    const u64 mag = v >= 0 ? (u64)v : (u64)(-(v + 1)) + 1; // |v| without overflow
    // |v| mod q by REDC(|v| * 2^64 mod q)
    const u64 r = redc(__umul64hi(mag, m.r1), mag * m.r1, m.q, m.qneg_inv);
    out[idx] = (v >= 0 || r == 0) ? r : m.q - r;
}

inline unsigned nblk(u64 n) { return (unsigned)((n + TPB - 1) / TPB); }

// device array of modulus indices 0..n-1 (cached per context size)
struct ModList {
    DevMem mem;
    u32 n = 0;
};

int mod_list(fheon_ctx *ctx, DevMem &m, u32 n)
{
    std::vector<u32> h(n);
    for (u32 i = 0; i < n; i++) h[i] = i;
    if (!m.alloc(n * sizeof(u32), ctx->stream)) return fail(ctx, FHEON_ERR_OOM, "modulus list");
    FHEON_CUDA(ctx, cudaMemcpyAsync(m.p, h.data(), n * sizeof(u32), cudaMemcpyHostToDevice, ctx->stream));
    FHEON_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return FHEON_OK;
}
} // namespace

int keygen_dev(fheon_ctx *ctx, fheon_sk *sk, fheon_pk *pk)
{
    const u32 N = ctx->N, L = ctx->L, n = ctx->L + ctx->K;
    cudaStream_t st = ctx->stream;
    const ModConst *mc = ctx->tab.mc.as<ModConst>();
    DevMem mods;
    int rc = mod_list(ctx, mods, n);
    if (rc) return rc;
    if (!sk->s.alloc((size_t)n * ctx->limb_bytes(), st) || !pk->b.alloc((size_t)2 * L * ctx->limb_bytes(), st))
        return fail(ctx, FHEON_ERR_OOM, "key allocation");
    u64 *s = sk->s.as<u64>();
    small_kernel<false><<<dim3(nblk(N / 8), 1), TPB, 0, st>>>(ctx->seed, DOM_SK, 0, 0, s, 0, N, mods.as<u32>(), n,
                                                              ctx->tab.cdt.as<u64>(), mc);
    FHEON_CUDA(ctx, cudaGetLastError());
    FHEON_CUDA(ctx, ntt_fwd_limbs(ctx, s, s, n, n, 0, st));
    u64 *pb = pk->b.as<u64>(), *pa = pb + (u64)L * N;
    uniform_kernel<<<dim3(nblk(N / 4), 1, L), TPB, 0, st>>>(ctx->seed, DOM_PK_A, 0, 0, 1, pa, 0, N, mods.as<u32>(), mc);
    small_kernel<true><<<dim3(nblk(N / 8), 1), TPB, 0, st>>>(ctx->seed, DOM_PK_E, 0, 0, pb, 0, N, mods.as<u32>(), L,
                                                             ctx->tab.cdt.as<u64>(), mc);
    FHEON_CUDA(ctx, cudaGetLastError());
    FHEON_CUDA(ctx, ntt_fwd_limbs(ctx, pb, pb, L, L, 0, st));
    key_combine_kernel<<<nblk((u64)L * N), TPB, 0, st>>>(pb, pa, s, nullptr, L, ctx->logN, -1, ctx->alpha, L,
                                                         ctx->tab.pmod.as<ulonglong2>(), mc, 0);
    FHEON_CUDA(ctx, cudaGetLastError());
    FHEON_CUDA(ctx, cudaStreamSynchronize(st)); // temporaries are released on return
    return FHEON_OK;
}

int galois_key_dev(fheon_ctx *ctx, const fheon_sk *sk, u64 g, RotKey &key)
{
    const u32 N = ctx->N, L = ctx->L, n = ctx->L + ctx->K, B = ctx->beta;
    cudaStream_t st = ctx->stream;
    const ModConst *mc = ctx->tab.mc.as<ModConst>();
    const size_t per = (size_t)n * N;
    DevMem mods, sg;
    int rc = mod_list(ctx, mods, n);
    if (rc) return rc;
    if (!key.mem.alloc((size_t)B * 2 * per * 8, st) || !sg.alloc(per * 8, st))
        return fail(ctx, FHEON_ERR_OOM, "rotation key allocation (%zu bytes)", (size_t)B * 2 * per * 8);
    u64 *k = key.mem.as<u64>();
    const u64 *s = sk->s.as<u64>();
    // the source key: sigma_g(s) for a rotation, s^2 for relinearisation (g = 0)
    if (g)
        gather_kernel<<<nblk(per), TPB, 0, st>>>(s, sg.as<u64>(), g, n, ctx->logN);
    else
        square_kernel<<<nblk(per), TPB, 0, st>>>(s, sg.as<u64>(), n, ctx->logN, mc);
    // e_j into the b slots (stream idx g<<32 | j<<16), a_j into the a slots
    // (stream idx g<<32 | j<<16 | limb)
    small_kernel<true><<<dim3(nblk(N / 8), B), TPB, 0, st>>>(ctx->seed, DOM_KSK_E, g << 32, 1ull << 16, k, 2 * per, N,
                                                             mods.as<u32>(), n, ctx->tab.cdt.as<u64>(), mc);
    uniform_kernel<<<dim3(nblk(N / 4), B, n), TPB, 0, st>>>(ctx->seed, DOM_KSK_A, g << 32, 1ull << 16, 1, k + per,
                                                            2 * per, N, mods.as<u32>(), mc);
    FHEON_CUDA(ctx, cudaGetLastError());
    for (u32 j = 0; j < B; j++) {
        u64 *b = k + (size_t)j * 2 * per, *a = b + per;
        FHEON_CUDA(ctx, ntt_fwd_limbs(ctx, b, b, n, n, 0, st));
        key_combine_kernel<<<nblk(per), TPB, 0, st>>>(b, a, s, sg.as<u64>(), n, ctx->logN, (int)j, ctx->alpha, L,
                                                      ctx->tab.pmod.as<ulonglong2>(), mc, 1);
        FHEON_CUDA(ctx, cudaGetLastError());
    }
    FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    return FHEON_OK;
}

cudaError_t key_from_mont(fheon_ctx *ctx, const u64 *in, u64 *out, size_t limbs_per_block, u32 blocks)
{
    const u64 total = (u64)limbs_per_block * blocks * ctx->N;
    from_mont_kernel<<<nblk(total), TPB, 0, ctx->stream>>>(in, out, (u32)limbs_per_block, total, ctx->logN,
                                                           ctx->tab.mc.as<ModConst>());
    return cudaGetLastError();
}

cudaError_t key_to_mont(fheon_ctx *ctx, u64 *x, size_t limbs_per_block, u32 blocks)
{
    const u64 total = (u64)limbs_per_block * blocks * ctx->N;
    to_mont_kernel<<<nblk(total), TPB, 0, ctx->stream>>>(x, (u32)limbs_per_block, total, ctx->logN,
                                                         ctx->tab.mc.as<ModConst>());
    return cudaGetLastError();
}

int encrypt_dev(fheon_ctx *ctx, const fheon_pk *pk, const fheon_pt *pt, u64 nonce, fheon_ct *out)
{
    const u32 N = ctx->N, L = ctx->L;
    cudaStream_t st = ctx->stream;
    const ModConst *mc = ctx->tab.mc.as<ModConst>();
    DevMem mods, tmp;
    int rc = mod_list(ctx, mods, L);
    if (rc) return rc;
    if (!tmp.alloc((size_t)3 * L * ctx->limb_bytes(), st)) return fail(ctx, FHEON_ERR_OOM, "encryption temporaries");
    rc = ct_reshape(ctx, out, L);
    if (rc) return rc;
    u64 *v = tmp.as<u64>(), *e0 = v + (u64)L * N, *e1 = e0 + (u64)L * N;
    small_kernel<false><<<dim3(nblk(N / 8), 1), TPB, 0, st>>>(ctx->seed, DOM_ENC_V, nonce, 0, v, 0, N, mods.as<u32>(),
                                                              L, ctx->tab.cdt.as<u64>(), mc);
    small_kernel<true><<<dim3(nblk(N / 8), 1), TPB, 0, st>>>(ctx->seed, DOM_ENC_E0, nonce, 0, e0, 0, N,
                                                             mods.as<u32>(), L, ctx->tab.cdt.as<u64>(), mc);
    small_kernel<true><<<dim3(nblk(N / 8), 1), TPB, 0, st>>>(ctx->seed, DOM_ENC_E1, nonce, 0, e1, 0, N,
                                                             mods.as<u32>(), L, ctx->tab.cdt.as<u64>(), mc);
    FHEON_CUDA(ctx, cudaGetLastError());
    // three polynomials of L limbs, each limb t under modulus q_t
    {
        MapParams mp = map_params(ctx, v, v, L, 0, L);
        FHEON_CUDA(ctx, (ntt::launch<false, MapJob>(ctx->logN, mp, 3 * L, st)));
    }
    encrypt_combine_kernel<<<nblk((u64)L * N), TPB, 0, st>>>(v, e0, e1, pk->b.as<u64>(), pt->m.as<u64>(), out->c0(), L,
                                                             ctx->logN, mc);
    FHEON_CUDA(ctx, cudaGetLastError());
    FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    return FHEON_OK;
}

int limbs_from_coeffs_dev(fheon_ctx *ctx, const long long *dev_coeffs, u32 level, u64 *out)
{
    cudaStream_t st = ctx->stream;
    coeffs_to_limbs_kernel<<<nblk((u64)level * ctx->N), TPB, 0, st>>>(dev_coeffs, out, level, ctx->logN,
                                                                      ctx->tab.mc.as<ModConst>());
    FHEON_CUDA(ctx, cudaGetLastError());
    FHEON_CUDA(ctx, ntt_fwd_limbs(ctx, out, out, level, level, 0, st));
    return FHEON_OK;
}

int plain_from_coeffs_dev(fheon_ctx *ctx, const int64_t *host_coeffs, u32 level, fheon_pt *pt)
{
    const u32 N = ctx->N;
    cudaStream_t st = ctx->stream;
    DevMem c;
    if (!c.alloc((size_t)N * 8, st) || !pt->m.alloc((size_t)level * ctx->limb_bytes(), st))
        return fail(ctx, FHEON_ERR_OOM, "plaintext allocation");
    FHEON_CUDA(ctx, cudaMemcpyAsync(c.p, host_coeffs, (size_t)N * 8, cudaMemcpyHostToDevice, st));
    int rc = limbs_from_coeffs_dev(ctx, c.as<long long>(), level, pt->m.as<u64>());
    if (rc) return rc;
    FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    return FHEON_OK;
}

} // namespace fheon
