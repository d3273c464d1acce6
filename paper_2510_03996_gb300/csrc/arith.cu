// arith.cu -- slot-wise ciphertext arithmetic around the rotation: plaintext
// products and sums (paper Sec. 5.1, kernel-vector products and their sum),
// decryption, and floor rescaling by the last prime (paper Sec. 6, depth).
// All are HBM-bound streams over u64[2][l][N]; each thread handles two
// adjacent coefficients with 16-byte accesses.
#include <algorithm>

#include "jobs.cuh"

namespace fheon {

namespace {
constexpr int TPB = 256;

__device__ __forceinline__ u32 limb_of(u64 idx, u32 level, u32 logN) { return (u32)((idx >> logN) % level); }

// out[b][i][n] = ct[b][i][n] * pt[i][n]
__global__ void __launch_bounds__(TPB) mul_plain_kernel(const u64 *__restrict__ ct, const u64 *__restrict__ pt,
                                                        u64 *__restrict__ out, u32 level, u32 logN,
                                                        const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= 2 * per) return;
    const u64 w = idx % per;
    const ModConst m = mc[(u32)(w >> logN)];
    const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ct + idx);
    const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(pt + w);
    *reinterpret_cast<ulonglong2 *>(out + idx) = make_ulonglong2(mulmod_plain(x.x, y.x, m), mulmod_plain(x.y, y.y, m));
}

// out (+)= sum_t ct_t * pt_t over both components: the products of up to 8
// terms are summed in 128 bits (8 q^2 < q 2^64 for every q < 2^61) and
// REDC'd, giving (sum) * 2^-64 mod q; the chunk results are added mod q and
// multiplied back by 2^64 mod q once.  Exact, so the result equals the
// sequence of plaintext products and additions it replaces.
struct MacArgs {
    const u64 *ct[MAC_MAX]; // u64[2][level][N]
    const u64 *pt[MAC_MAX]; // u64[>= level][N]
};
__global__ void __launch_bounds__(TPB) mac_plain_kernel(const __grid_constant__ MacArgs A, u32 n, u64 *out, bool add_out,
                                                        u32 level, u32 logN, const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= 2 * per) return;
    const u64 w = idx % per;
    const ModConst m = mc[(u32)(w >> logN)];
    u64 s0 = 0, s1 = 0;
    for (u32 c = 0; c < n; c += 8) {
        u128acc a0, a1;
        acc_zero(a0);
        acc_zero(a1);
        const u32 e = min(n, c + 8);
        for (u32 t = c; t < e; t++) {
            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(A.ct[t] + idx);
            const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(A.pt[t] + w);
            acc_mad(a0, x.x, y.x);
            acc_mad(a1, x.y, y.y);
        }
        s0 = addmod(s0, redc_acc(a0, m.q, m.qneg_inv), m.q);
        s1 = addmod(s1, redc_acc(a1, m.q, m.qneg_inv), m.q);
    }
    s0 = shoup(s0, m.r1, m.r1_sh, m.q);
    s1 = shoup(s1, m.r1, m.r1_sh, m.q);
    if (add_out) {
        const ulonglong2 o = *reinterpret_cast<const ulonglong2 *>(out + idx);
        s0 = addmod(s0, o.x, m.q);
        s1 = addmod(s1, o.y, m.q);
    }
    *reinterpret_cast<ulonglong2 *>(out + idx) = make_ulonglong2(s0, s1);
}

// several groups' sums over one set of taps: outs[g] = sum_t ct_t * pt[g][t].
// A block is GB groups x (TPB / GB) coefficient pairs: each warp sums one
// group over 32 consecutive pairs (the same per-thread work as
// mac_plain_kernel, coalesced), and the GB warps of a block that read the
// same tap coefficients share them through L1, so the taps cross HBM about
// once per GB groups instead of once per group.  Measured on a 64-channel
// ResNet-20 convolution at N = 2^16 (45 taps, 26 groups, level 11): GB = 4
// takes 3.34 ms (2: 3.53, 8: 3.40) against 4.70 ms group by group; one thread
// holding the sums of two groups took 4.06 ms, of four or eight (78 and 128
// registers a thread) 4.86 and 6.50 ms.
struct MacGroupArgs {
    const u64 *ct[MACG_TAPS];              // u64[2][level][N]
    const u64 *pt[MACG_GROUPS][MACG_TAPS]; // u64[>= level][N]; null: no product
    u64 *out[MACG_GROUPS];
};
template <u32 GB>
__global__ void __launch_bounds__(TPB) mac_groups_kernel(const __grid_constant__ MacGroupArgs A, u32 nt, u32 ng,
                                                         u32 level, u32 logN, const ModConst *__restrict__ mc)
{
    // the block's pointers in shared memory (indexed by tap and group, the
    // parameter bank's cache would serialise)
    __shared__ const u64 *sct[MACG_TAPS];
    __shared__ const u64 *spt[GB][MACG_TAPS];
    const u32 g0 = blockIdx.y * GB;
    for (u32 i = threadIdx.x; i < nt; i += TPB) sct[i] = A.ct[i];
    for (u32 i = threadIdx.x; i < GB * nt; i += TPB)
        spt[i / nt][i % nt] = g0 + i / nt < ng ? A.pt[g0 + i / nt][i % nt] : nullptr;
    __syncthreads();
    constexpr u32 PAIRS = TPB / GB;
    const u32 k = threadIdx.x / PAIRS;
    const u64 idx = ((u64)blockIdx.x * PAIRS + threadIdx.x % PAIRS) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= 2 * per || g0 + k >= ng) return;
    const u64 w = idx % per;
    const ModConst m = mc[(u32)(w >> logN)];
    u64 s0 = 0, s1 = 0;
    u128acc a0, a1;
    acc_zero(a0);
    acc_zero(a1);
    u32 cnt = 0;
    for (u32 t = 0; t < nt; t++) {
        const u64 *p = spt[k][t];
        if (!p) continue;
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(sct[t] + idx);
        const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(p + w);
        acc_mad(a0, x.x, y.x);
        acc_mad(a1, x.y, y.y);
        if (++cnt == 8) { // at most 8 products between reductions (8 q^2 < q 2^64)
            s0 = addmod(s0, redc_acc(a0, m.q, m.qneg_inv), m.q);
            s1 = addmod(s1, redc_acc(a1, m.q, m.qneg_inv), m.q);
            acc_zero(a0);
            acc_zero(a1);
            cnt = 0;
        }
    }
    s0 = addmod(s0, redc_acc(a0, m.q, m.qneg_inv), m.q);
    s1 = addmod(s1, redc_acc(a1, m.q, m.qneg_inv), m.q);
    s0 = shoup(s0, m.r1, m.r1_sh, m.q);
    s1 = shoup(s1, m.r1, m.r1_sh, m.q);
    *reinterpret_cast<ulonglong2 *>(A.out[g0 + k] + idx) = make_ulonglong2(s0, s1);
}

// the ciphertext tensor d = (a0 b0, a0 b1 + a1 b0, a1 b1) over the lowest
// `level` limbs of each component (components may sit at any stride, so an
// operand at a higher level is read in place); the middle term's two
// products summed in 128 bits and reduced once; `twice` doubles all three
// (the tensor of 2a and b)
__global__ void __launch_bounds__(TPB) tensor_kernel(const u64 *__restrict__ a0p, const u64 *__restrict__ a1p,
                                                     const u64 *__restrict__ b0p, const u64 *__restrict__ b1p,
                                                     u64 *__restrict__ d, u32 level, bool twice, u32 logN,
                                                     const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= per) return;
    const ModConst m = mc[(u32)(idx >> logN)];
    const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(a0p + idx), a1 = *reinterpret_cast<const ulonglong2 *>(a1p + idx);
    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(b0p + idx), b1 = *reinterpret_cast<const ulonglong2 *>(b1p + idx);
    u128acc x, y;
    acc_zero(x);
    acc_zero(y);
    acc_mad(x, a0.x, b1.x);
    acc_mad(x, a1.x, b0.x);
    acc_mad(y, a0.y, b1.y);
    acc_mad(y, a1.y, b0.y);
    u64 r[6] = {mulmod_plain(a0.x, b0.x, m), mulmod_plain(a0.y, b0.y, m),
                shoup(redc_acc(x, m.q, m.qneg_inv), m.r1, m.r1_sh, m.q), shoup(redc_acc(y, m.q, m.qneg_inv), m.r1, m.r1_sh, m.q),
                mulmod_plain(a1.x, b1.x, m), mulmod_plain(a1.y, b1.y, m)};
    if (twice) {
#pragma unroll
        for (int i = 0; i < 6; i++) r[i] = addmod(r[i], r[i], m.q);
    }
    *reinterpret_cast<ulonglong2 *>(d + idx) = make_ulonglong2(r[0], r[1]);
    *reinterpret_cast<ulonglong2 *>(d + per + idx) = make_ulonglong2(r[2], r[3]);
    *reinterpret_cast<ulonglong2 *>(d + 2 * per + idx) = make_ulonglong2(r[4], r[5]);
}

// v mod q for a signed 64-bit v: REDC(v) = v 2^-64 mod q (v < q 2^64), then
// a Montgomery product with 2^128 mod q restores v mod q
__device__ __forceinline__ u64 signed_mod(long long v, const ModConst &m)
{
    const u64 a = v >= 0 ? (u64)v : (u64)(-(v + 1)) + 1ull; // |v|, also for INT64_MIN
    const u64 r = mulmod_mont(redc(0, a, m.q, m.qneg_inv), m.r2, m);
    return (v >= 0 || r == 0) ? r : m.q - r;
}

// out = v * ct over `ncomp` components of `level` limbs; input component c at
// ct + c * in_stride (in_stride = level * N for a ciphertext at this level)
__global__ void __launch_bounds__(TPB) mul_int_kernel(const u64 *__restrict__ ct, u64 in_stride, long long v,
                                                      u64 *__restrict__ out, u32 level, u32 ncomp, u32 logN,
                                                      const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= ncomp * per) return;
    const ModConst m = mc[limb_of(idx, level, logN)];
    const u64 vm = signed_mod(v, m);
    const u64 comp = idx / per;
    const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ct + comp * in_stride + (idx - comp * per));
    *reinterpret_cast<ulonglong2 *>(out + idx) = make_ulonglong2(mulmod_plain(x.x, vm, m), mulmod_plain(x.y, vm, m));
}

// out = ct + v: the constant polynomial v is v at every evaluation point, so
// component 0 gains v mod q_i everywhere; component 1 is copied
__global__ void __launch_bounds__(TPB) add_int_kernel(const u64 *__restrict__ ct, long long v, u64 *__restrict__ out,
                                                      u32 level, u32 logN, const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= 2 * per) return;
    ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ct + idx);
    if (idx < per) {
        const ModConst m = mc[(u32)(idx >> logN)];
        const u64 vm = signed_mod(v, m);
        x = make_ulonglong2(addmod(x.x, vm, m.q), addmod(x.y, vm, m.q));
    }
    *reinterpret_cast<ulonglong2 *>(out + idx) = x;
}

// out (+)= sum_t K_t * ct_t over both components, each ct_t read at its own
// component stride (its lowest `level` limbs); the constants reduced per
// modulus, the products summed in 128 bits in chunks of 8 as in
// mac_plain_kernel
struct LinArgs {
    const u64 *ct[MAC_MAX];
    u64 stride[MAC_MAX];
    long long K[MAC_MAX];
};
__global__ void __launch_bounds__(TPB) lincomb_kernel(const __grid_constant__ LinArgs A, u32 n, u64 *out, bool add_out,
                                                      u32 level, u32 logN, const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= 2 * per) return;
    const u64 comp = idx / per, w = idx - comp * per;
    const ModConst m = mc[(u32)(w >> logN)];
    u64 s0 = 0, s1 = 0;
    for (u32 c = 0; c < n; c += 8) {
        u128acc a0, a1;
        acc_zero(a0);
        acc_zero(a1);
        const u32 e = min(n, c + 8);
        for (u32 t = c; t < e; t++) {
            const u64 k = signed_mod(A.K[t], m);
            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(A.ct[t] + comp * A.stride[t] + w);
            acc_mad(a0, x.x, k);
            acc_mad(a1, x.y, k);
        }
        s0 = addmod(s0, redc_acc(a0, m.q, m.qneg_inv), m.q);
        s1 = addmod(s1, redc_acc(a1, m.q, m.qneg_inv), m.q);
    }
    s0 = shoup(s0, m.r1, m.r1_sh, m.q);
    s1 = shoup(s1, m.r1, m.r1_sh, m.q);
    if (add_out) {
        const ulonglong2 o = *reinterpret_cast<const ulonglong2 *>(out + idx);
        s0 = addmod(s0, o.x, m.q);
        s1 = addmod(s1, o.y, m.q);
    }
    *reinterpret_cast<ulonglong2 *>(out + idx) = make_ulonglong2(s0, s1);
}

// out = a + b over `ncomp` components of `level` limbs
__global__ void __launch_bounds__(TPB) add_kernel(const u64 *__restrict__ a, const u64 *__restrict__ b,
                                                  u64 *__restrict__ out, u32 level, u32 ncomp, u32 logN,
                                                  const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    if (idx >= ((u64)ncomp * level << logN)) return;
    const u64 q = mc[limb_of(idx, level, logN)].q;
    const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(a + idx);
    const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(b + idx);
    *reinterpret_cast<ulonglong2 *>(out + idx) = make_ulonglong2(addmod(x.x, y.x, q), addmod(x.y, y.y, q));
}

// out = (c0 + pt, c1)
__global__ void __launch_bounds__(TPB) add_plain_kernel(const u64 *__restrict__ ct, const u64 *__restrict__ pt,
                                                        u64 *__restrict__ out, u32 level, u32 logN,
                                                        const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= 2 * per) return;
    const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ct + idx);
    ulonglong2 r = x;
    if (idx < per) {
        const u64 q = mc[(u32)(idx >> logN)].q;
        const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(pt + idx);
        r = make_ulonglong2(addmod(x.x, y.x, q), addmod(x.y, y.y, q));
    }
    *reinterpret_cast<ulonglong2 *>(out + idx) = r;
}

// m = c0 + c1 * s
__global__ void __launch_bounds__(TPB) decrypt_kernel(const u64 *__restrict__ ct, const u64 *__restrict__ s,
                                                      u64 *__restrict__ m, u32 level, u32 logN,
                                                      const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u64 per = (u64)level << logN;
    if (idx >= per) return;
    const ModConst c = mc[(u32)(idx >> logN)];
    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(ct + idx);
    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(ct + per + idx);
    const ulonglong2 k = *reinterpret_cast<const ulonglong2 *>(s + idx);
    *reinterpret_cast<ulonglong2 *>(m + idx) =
        make_ulonglong2(addmod(a.x, mulmod_plain(b.x, k.x, c), c.q), addmod(a.y, mulmod_plain(b.y, k.y, c), c.q));
}

// out[b][i] = (x[b][i] - y[b][i]) * q_t^-1 mod q_i, i < level-1 (x over `level` limbs)
__global__ void __launch_bounds__(TPB) rescale_combine_kernel(const u64 *__restrict__ x, const u64 *__restrict__ y,
                                                              u64 *__restrict__ out, u32 level, u32 logN, u32 L,
                                                              const ulonglong2 *__restrict__ rinv,
                                                              const ModConst *__restrict__ mc)
{
    const u64 idx = ((u64)blockIdx.x * TPB + threadIdx.x) * 2;
    const u32 lo = level - 1;
    const u64 per = (u64)lo << logN;
    if (idx >= 2 * per) return;
    const u32 b = (u32)(idx / per);
    const u64 w = idx % per;
    const u32 i = (u32)(w >> logN);
    const u64 q = mc[i].q;
    const ulonglong2 f = rinv[(u64)lo * L + i];
    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(x + (u64)b * ((u64)level << logN) + w);
    const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(y + idx);
    *reinterpret_cast<ulonglong2 *>(out + idx) =
        make_ulonglong2(shoup(a.x + q - c.x, f.x, f.y, q), shoup(a.y + q - c.y, f.x, f.y, q));
}

// Forward NTT of [x]_{q_t} reduced into each q_i: limb position p of polynomial
// b reads the coefficients of b's last limb (any value < 2^64 reduces exactly:
// REDC(x * (2^64 mod q)) = x mod q).
struct ReduceLoadJob : MapJob {
    using Params = MapParams;
    __device__ ReduceLoadJob(const MapParams &P, u32 job) : MapJob(P, job)
    {
        in = P.in + (job / P.per_poly) * P.in_poly_stride; // same source limb for every i
    }
    template <bool INV> __device__ u64 load_first(u32 J) const
    {
        const ModConst m = p.tp.mc[midx];
        const u64 v = in[J];
        return redc(__umul64hi(v, m.r1), v * m.r1, m.q, m.qneg_inv);
    }
};

// Forward NTT of the centred lift of [x]_{q_0} into each q_i (ModRaise):
// coefficients above q_0 / 2 stand for x - q_0, whose residue is
// x mod q_i - q_0 mod q_i (both reduced by REDC(v * (2^64 mod q_i))).
struct CenterLoadJob : MapJob {
    using Params = MapParams;
    __device__ CenterLoadJob(const MapParams &P, u32 job) : MapJob(P, job)
    {
        in = P.in + (job / P.per_poly) * P.in_poly_stride;
    }
    template <bool INV> __device__ u64 load_first(u32 J) const
    {
        const ModConst m = p.tp.mc[midx];
        const u64 q0 = p.tp.mc[0].q;
        const u64 v = in[J];
        const u64 r = redc(__umul64hi(v, m.r1), v * m.r1, m.q, m.qneg_inv);
        if (v <= (q0 >> 1)) return r;
        const u64 c = redc(__umul64hi(q0, m.r1), q0 * m.r1, m.q, m.qneg_inv);
        return r >= c ? r - c : r + m.q - c;
    }
};

inline unsigned blocks2(u64 elems) { return (unsigned)((elems / 2 + TPB - 1) / TPB); }
} // namespace

cudaError_t k_mul_plain(fheon_ctx *ctx, const u64 *ct, const u64 *pt, u64 *out, u32 level, u32)
{
    mul_plain_kernel<<<blocks2((u64)2 * level * ctx->N), TPB, 0, ctx->stream>>>(ct, pt, out, level, ctx->logN,
                                                                                ctx->tab.mc.as<ModConst>());
    prof_mark(ctx->stream, "mul_plain");
    return cudaGetLastError();
}
cudaError_t k_mac_plain(fheon_ctx *ctx, const u64 *const *cts, const u64 *const *pts, u32 n, u64 *out, u32 level)
{
    for (u32 s = 0; s < n; s += MAC_MAX) {
        MacArgs A{};
        const u32 m = std::min<u32>(MAC_MAX, n - s);
        for (u32 t = 0; t < m; t++) {
            A.ct[t] = cts[s + t];
            A.pt[t] = pts[s + t];
        }
        mac_plain_kernel<<<blocks2((u64)2 * level * ctx->N), TPB, 0, ctx->stream>>>(A, m, out, s > 0, level, ctx->logN,
                                                                                     ctx->tab.mc.as<ModConst>());
        prof_mark(ctx->stream, "mac_plain");
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t k_mac_groups(fheon_ctx *ctx, const u64 *const *cts, u32 nt, const u64 *const *pts, u32 ng,
                         u64 *const *outs, u32 level)
{
    if (nt == 0 || nt > MACG_TAPS || ng == 0 || ng > MACG_GROUPS) return cudaErrorInvalidValue;
    MacGroupArgs A{};
    for (u32 t = 0; t < nt; t++) A.ct[t] = cts[t];
    for (u32 g = 0; g < ng; g++) {
        A.out[g] = outs[g];
        for (u32 t = 0; t < nt; t++) A.pt[g][t] = pts[(size_t)g * nt + t];
    }
    {
        constexpr u32 GB = MACG_BLOCK_GROUPS;
        const u64 pairs = (u64)level * ctx->N;
        const dim3 grid((unsigned)((pairs + TPB / GB - 1) / (TPB / GB)), (ng + GB - 1) / GB);
        mac_groups_kernel<GB><<<grid, TPB, 0, ctx->stream>>>(A, nt, ng, level, ctx->logN, ctx->tab.mc.as<ModConst>());
        prof_mark(ctx->stream, "mac_groups");
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t k_tensor(fheon_ctx *ctx, const u64 *a0, const u64 *a1, const u64 *b0, const u64 *b1, u64 *d, u32 level,
                     bool twice)
{
    tensor_kernel<<<blocks2((u64)level * ctx->N), TPB, 0, ctx->stream>>>(a0, a1, b0, b1, d, level, twice, ctx->logN,
                                                                          ctx->tab.mc.as<ModConst>());
    prof_mark(ctx->stream, "tensor");
    return cudaGetLastError();
}
cudaError_t k_mul_int(fheon_ctx *ctx, const u64 *ct, int64_t v, u64 *out, u32 level, u32 ncomp, u64 in_stride)
{
    if (!in_stride) in_stride = (u64)level * ctx->N;
    mul_int_kernel<<<blocks2((u64)ncomp * level * ctx->N), TPB, 0, ctx->stream>>>(ct, in_stride, (long long)v, out, level,
                                                                                  ncomp, ctx->logN,
                                                                                  ctx->tab.mc.as<ModConst>());
    prof_mark(ctx->stream, "mul_int");
    return cudaGetLastError();
}
cudaError_t k_add_int(fheon_ctx *ctx, const u64 *ct, int64_t v, u64 *out, u32 level)
{
    add_int_kernel<<<blocks2((u64)2 * level * ctx->N), TPB, 0, ctx->stream>>>(ct, (long long)v, out, level, ctx->logN,
                                                                               ctx->tab.mc.as<ModConst>());
    prof_mark(ctx->stream, "add_int");
    return cudaGetLastError();
}
cudaError_t k_lincomb(fheon_ctx *ctx, const u64 *const *cts, const u64 *strides, const int64_t *K, u32 n, u64 *out,
                      u32 level)
{
    for (u32 s = 0; s < n; s += MAC_MAX) {
        LinArgs A{};
        const u32 m = std::min<u32>(MAC_MAX, n - s);
        for (u32 t = 0; t < m; t++) {
            A.ct[t] = cts[s + t];
            A.stride[t] = strides[s + t];
            A.K[t] = (long long)K[s + t];
        }
        lincomb_kernel<<<blocks2((u64)2 * level * ctx->N), TPB, 0, ctx->stream>>>(A, m, out, s > 0, level, ctx->logN,
                                                                                   ctx->tab.mc.as<ModConst>());
        prof_mark(ctx->stream, "lincomb");
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t k_add(fheon_ctx *ctx, const u64 *a, const u64 *b, u64 *out, u32 level, u32 ncomp)
{
    add_kernel<<<blocks2((u64)ncomp * level * ctx->N), TPB, 0, ctx->stream>>>(a, b, out, level, ncomp, ctx->logN,
                                                                              ctx->tab.mc.as<ModConst>());
    prof_mark(ctx->stream, "add");
    return cudaGetLastError();
}
cudaError_t k_add_plain(fheon_ctx *ctx, const u64 *ct, const u64 *pt, u64 *out, u32 level)
{
    add_plain_kernel<<<blocks2((u64)2 * level * ctx->N), TPB, 0, ctx->stream>>>(ct, pt, out, level, ctx->logN,
                                                                                ctx->tab.mc.as<ModConst>());
    prof_mark(ctx->stream, "add_plain");
    return cudaGetLastError();
}
cudaError_t k_decrypt(fheon_ctx *ctx, const u64 *ct, const u64 *s, u64 *m, u32 level)
{
    decrypt_kernel<<<blocks2((u64)level * ctx->N), TPB, 0, ctx->stream>>>(ct, s, m, level, ctx->logN,
                                                                          ctx->tab.mc.as<ModConst>());
    return cudaGetLastError();
}

cudaError_t ntt_fwd_limbs(fheon_ctx *ctx, const u64 *in, u64 *out, u32 n, u32 level, u32 first_limb, cudaStream_t st)
{
    MapParams mp = map_params(ctx, in, out, n, first_limb, level);
    return ntt::launch<false, MapJob>(ctx->logN, mp, n, st);
}
cudaError_t ntt_inv_limbs(fheon_ctx *ctx, const u64 *in, u64 *out, u32 n, u32 level, u32 first_limb, cudaStream_t st)
{
    MapParams mp = map_params(ctx, in, out, n, first_limb, level);
    return ntt::launch<true, MapJob>(ctx->logN, mp, n, st);
}

int mod_raise_ct(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out)
{
    const u32 L = ctx->L, N = ctx->N;
    int rc = ensure_workspace(ctx, ctx->ks_ws_limbs(ctx->L) + 2 * (size_t)ctx->L);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    u64 *x0 = ctx->ws.as<u64>(); // [2][N] coefficients mod q_0
    {
        MapParams mp = map_params(ctx, in->c0(), x0, 1, 0, 1);
        mp.in_poly_stride = (u64)in->level * N;
        mp.out_poly_stride = N;
        FHEON_CUDA(ctx, (ntt::launch<true, MapJob>(ctx->logN, mp, 2, st)));
    }
    if ((rc = ct_reshape(ctx, out, L))) return rc;
    {
        MapParams mp = map_params(ctx, x0, out->c0(), L, 0, L);
        mp.in_poly_stride = N;
        mp.out_poly_stride = (u64)L * N;
        FHEON_CUDA(ctx, (ntt::launch<false, CenterLoadJob>(ctx->logN, mp, 2 * L, st)));
    }
    prof_mark(st, "mod_raise");
    return FHEON_OK;
}

int rescale_ct(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out)
{
    const u32 l = in->level, N = ctx->N, t = l - 1;
    const size_t need = 2 + (size_t)2 * t + 2 * (size_t)t; // last-limb coeffs, y, staging
    int rc = ensure_workspace(ctx, need > ctx->ks_ws_limbs(ctx->L) + 2 * (size_t)ctx->L
                                       ? need
                                       : ctx->ks_ws_limbs(ctx->L) + 2 * (size_t)ctx->L);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    u64 *xl = ctx->ws.as<u64>();       // [2][N] coefficients of the last limb
    u64 *y = xl + (u64)2 * N;          // [2][t][N]
    u64 *stage = y + (u64)2 * t * N;   // [2][t][N]
    // INTT of the last limb of c0 and c1 (modulus q_t)
    {
        MapParams mp = map_params(ctx, in->c0() + (u64)t * N, xl, 1, t, l);
        mp.in_poly_stride = (u64)l * N;
        mp.out_poly_stride = N;
        FHEON_CUDA(ctx, (ntt::launch<true, MapJob>(ctx->logN, mp, 2, st)));
    }
    // [x]_{q_t} into every q_i, i < t, forward NTT
    {
        MapParams mp = map_params(ctx, xl, y, t, 0, t);
        mp.in_poly_stride = N;
        mp.out_poly_stride = (u64)t * N;
        FHEON_CUDA(ctx, (ntt::launch<false, ReduceLoadJob>(ctx->logN, mp, 2 * t, st)));
    }
    const bool inplace = (out == in);
    u64 *dst = stage;
    if (!inplace) {
        rc = ct_reshape(ctx, out, t);
        if (rc) return rc;
        dst = out->c0();
    }
    const double sc = in->scale / (double)ctx->mod[t];
    rescale_combine_kernel<<<blocks2((u64)2 * t * N), TPB, 0, st>>>(in->c0(), y, dst, l, ctx->logN, ctx->L,
                                                                     ctx->tab.rescale_inv.as<ulonglong2>(),
                                                                     ctx->tab.mc.as<ModConst>());
    prof_mark(st, "rescale_combine");
    FHEON_CUDA(ctx, cudaGetLastError());
    if (inplace) {
        FHEON_CUDA(ctx, cudaMemcpyAsync(out->c0(), stage, (size_t)2 * t * ctx->limb_bytes(), cudaMemcpyDeviceToDevice, st));
        out->level = t;
    }
    out->scale = sc;
    return FHEON_OK;
}

} // namespace fheon
