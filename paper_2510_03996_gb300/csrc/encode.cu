// encode.cu -- CKKS encoding and decoding (paper Sec. 3.2: a vector of N/2
// complex slots maps to R = Z[X]/(X^N+1)), in FP64 on the device.
//
// Slot i is the evaluation at zeta^(5^i mod 2N), zeta = exp(i pi / N).  With
// n = N/2, u_k = m_k + i m_{k+n} and 5^i = 4 a_i + 1 (mod 2N):
//   z_i = sum_k m_k zeta^(5^i k) = DFT_n(u_k zeta^k)[a_i],  DFT_n with e^{+2 pi i/n},
// so decoding is a twist, one length-n complex FFT and the slot permutation
// a_i; encoding runs the same steps backwards and rounds
// m = round(scale * (Re u, Im u)) half away from zero.
#include <cmath>
#include <vector>

#include "jobs.cuh"

namespace fheon {

namespace {
constexpr int TPB = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// out[brv(k)] = in[k] over n = 2^logn entries
__global__ void bitrev_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, u32 logn)
{
    const u32 k = blockIdx.x * TPB + threadIdx.x;
    if (k >= (1u << logn)) return;
    out[__brev(k) >> (32 - logn)] = in[k];
}

// one radix-2 decimation-in-time stage with butterflies of half-size `half`;
// sign = +1: e^{+2 pi i/n} twiddles, -1: conjugates
__global__ void fft_stage_kernel(double2 *x, const double2 *__restrict__ w, u32 logn, u32 half, int sign)
{
    const u32 b = blockIdx.x * TPB + threadIdx.x;
    const u32 n = 1u << logn;
    if (b >= n / 2) return;
    const u32 pos = b & (half - 1), grp = b / half;
    const u32 i = grp * 2 * half + pos, j = i + half;
    double2 tw = w[pos * (n / (2 * half))];
    if (sign < 0) tw.y = -tw.y;
    const double2 t = cmul(tw, x[j]);
    const double2 a = x[i];
    x[i] = make_double2(a.x + t.x, a.y + t.y);
    x[j] = make_double2(a.x - t.x, a.y - t.y);
}

// V[a_i] = z_i for i < nz, zero elsewhere
__global__ void slot_scatter_kernel(const double *__restrict__ re, const double *__restrict__ im,
                                    const u32 *__restrict__ perm, double2 *__restrict__ V, u32 nz, u32 n)
{
    const u32 i = blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    if (i < nz) V[perm[i]] = make_double2(re[i], im ? im[i] : 0.0);
}

// u_k = X_k / n * zeta^-k; m_k = round(scale Re u_k), m_{k+n} = round(scale Im u_k)
__global__ void encode_round_kernel(const double2 *__restrict__ X, const double2 *__restrict__ zeta,
                                    long long *__restrict__ m, u32 n, double scale, int *__restrict__ overflow)
{
    const u32 k = blockIdx.x * TPB + threadIdx.x;
    if (k >= n) return;
    double2 zc = zeta[k];
    zc.y = -zc.y;
    const double2 u = cmul(X[k], zc);
    const double f = scale / (double)n;
    const double a = round(u.x * f), b = round(u.y * f);
    const double lim = 4.611686018427387904e18; // 2^62
    if (!(fabs(a) < lim) || !(fabs(b) < lim)) {
        *overflow = 1;
        m[k] = 0;
        m[k + n] = 0;
        return;
    }
    m[k] = (long long)a;
    m[k + n] = (long long)b;
}

// centred lift of the lowest one or two limbs (coefficient form), divided by
// scale, packed as u_k = (m_k + i m_{k+n}) / scale, times zeta^k
__global__ void decode_lift_kernel(const u64 *__restrict__ c, u32 nlimb, u64 q0, u64 q1, u64 q0inv_mod_q1,
                                   u64 q0inv_sh, const double2 *__restrict__ zeta, double2 *__restrict__ u, u32 n,
                                   double inv_scale)
{
    const u32 k = blockIdx.x * TPB + threadIdx.x;
    if (k >= n) return;
    double v[2];
    for (int h = 0; h < 2; h++) {
        const u32 idx = k + h * n;
        const u64 r0 = c[idx];
        if (nlimb == 1) {
            v[h] = r0 > q0 / 2 ? -(double)(q0 - r0) : (double)r0;
            continue;
        }
        const u64 r1 = c[(u64)2 * n + idx];
        // x = r0 + q0 * ((r1 - r0) q0^-1 mod q1), 0 <= x < q0 q1 (CRT)
        const u64 d = (r1 >= r0 % q1) ? r1 - r0 % q1 : r1 + q1 - r0 % q1;
        const u64 tq = shoup(d, q0inv_mod_q1, q0inv_sh, q1);
        u64 lo = tq * q0, hi = __umul64hi(tq, q0);
        lo += r0;
        hi += (lo < r0) ? 1 : 0;
        // Q = q0*q1; centre: if x > Q/2 then x - Q
        const u64 Qlo = q0 * q1, Qhi = __umul64hi(q0, q1);
        const u64 hQlo = (Qlo >> 1) | (Qhi << 63), hQhi = Qhi >> 1;
        const bool big = (hi > hQhi) || (hi == hQhi && lo > hQlo);
        if (big) {
            const u64 nlo = Qlo - lo, nhi = Qhi - hi - (Qlo < lo ? 1 : 0);
            v[h] = -((double)nhi * 18446744073709551616.0 + (double)nlo);
        } else {
            v[h] = (double)hi * 18446744073709551616.0 + (double)lo;
        }
    }
    u[k] = cmul(make_double2(v[0] * inv_scale, v[1] * inv_scale), zeta[k]);
}

__global__ void slot_gather_kernel(const double2 *__restrict__ V, const u32 *__restrict__ perm,
                                   double *__restrict__ re, double *__restrict__ im, u32 nz)
{
    const u32 i = blockIdx.x * TPB + threadIdx.x;
    if (i >= nz) return;
    const double2 z = V[perm[i]];
    re[i] = z.x;
    if (im) im[i] = z.y;
}

inline unsigned nblk(u64 n) { return (unsigned)((n + TPB - 1) / TPB); }

cudaError_t fft(fheon_ctx *ctx, const double2 *in, double2 *out, int sign)
{
    const u32 logn = ctx->logN - 1, n = 1u << logn;
    bitrev_kernel<<<nblk(n), TPB, 0, ctx->stream>>>(in, out, logn);
    for (u32 half = 1; half < n; half <<= 1)
        fft_stage_kernel<<<nblk(n / 2), TPB, 0, ctx->stream>>>(out, ctx->tab.fft_w.as<double2>(), logn, half, sign);
    return cudaGetLastError();
}
} // namespace

int build_fft_tables(fheon_ctx *ctx)
{
    const u32 N = ctx->N, n = N / 2;
    std::vector<double2> w(n), z(n);
    std::vector<u32> perm(n);
    for (u32 j = 0; j < n; j++) {
        const double a = 2.0 * M_PI * (double)j / (double)n, b = M_PI * (double)j / (double)N;
        w[j] = make_double2(std::cos(a), std::sin(a));
        z[j] = make_double2(std::cos(b), std::sin(b));
    }
    u64 p = 1;
    for (u32 i = 0; i < n; i++) {
        perm[i] = (u32)((p - 1) / 4);
        p = p * 5 % (2ull * N);
    }
    cudaStream_t st = ctx->stream;
    if (!ctx->tab.fft_w.alloc(n * sizeof(double2), st) || !ctx->tab.fft_zeta.alloc(n * sizeof(double2), st) ||
        !ctx->tab.slot_perm.alloc(n * sizeof(u32), st))
        return fail(ctx, FHEON_ERR_OOM, "FFT tables");
    FHEON_CUDA(ctx, cudaMemcpyAsync(ctx->tab.fft_w.p, w.data(), n * sizeof(double2), cudaMemcpyHostToDevice, st));
    FHEON_CUDA(ctx, cudaMemcpyAsync(ctx->tab.fft_zeta.p, z.data(), n * sizeof(double2), cudaMemcpyHostToDevice, st));
    FHEON_CUDA(ctx, cudaMemcpyAsync(ctx->tab.slot_perm.p, perm.data(), n * sizeof(u32), cudaMemcpyHostToDevice, st));
    FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    return FHEON_OK;
}

int encode_dev(fheon_ctx *ctx, const double *re, const double *im, u32 nz, double scale, u32 level, fheon_pt *pt,
               int64_t *host_coeffs_out)
{
    const u32 N = ctx->N, n = N / 2;
    cudaStream_t st = ctx->stream;
    DevMem zin, V, X, m, flag;
    if (!zin.alloc((size_t)2 * n * 8, st) || !V.alloc((size_t)n * 16, st) || !X.alloc((size_t)n * 16, st) ||
        !m.alloc((size_t)N * 8, st) || !flag.alloc(sizeof(int), st))
        return fail(ctx, FHEON_ERR_OOM, "encode temporaries");
    double *dre = zin.as<double>(), *dim = dre + n;
    if (nz) {
        FHEON_CUDA(ctx, cudaMemcpyAsync(dre, re, (size_t)nz * 8, cudaMemcpyHostToDevice, st));
        if (im) FHEON_CUDA(ctx, cudaMemcpyAsync(dim, im, (size_t)nz * 8, cudaMemcpyHostToDevice, st));
    }
    FHEON_CUDA(ctx, cudaMemsetAsync(V.p, 0, (size_t)n * 16, st));
    FHEON_CUDA(ctx, cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    slot_scatter_kernel<<<nblk(n), TPB, 0, st>>>(dre, im ? dim : nullptr, ctx->tab.slot_perm.as<u32>(),
                                                 V.as<double2>(), nz, n);
    FHEON_CUDA(ctx, fft(ctx, V.as<double2>(), X.as<double2>(), -1));
    encode_round_kernel<<<nblk(n), TPB, 0, st>>>(X.as<double2>(), ctx->tab.fft_zeta.as<double2>(), m.as<long long>(),
                                                 n, scale, flag.as<int>());
    FHEON_CUDA(ctx, cudaGetLastError());
    int ovf = 0;
    FHEON_CUDA(ctx, cudaMemcpyAsync(&ovf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    if (ovf) return fail(ctx, FHEON_ERR_ARG, "encoded coefficient exceeds 2^62 (scale too large)");
    if (host_coeffs_out) {
        FHEON_CUDA(ctx, cudaMemcpyAsync(host_coeffs_out, m.p, (size_t)N * 8, cudaMemcpyDeviceToHost, st));
        FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    }
    if (pt) {
        if (!pt->m.alloc((size_t)level * ctx->limb_bytes(), st)) return fail(ctx, FHEON_ERR_OOM, "plaintext");
        int rc = limbs_from_coeffs_dev(ctx, m.as<long long>(), level, pt->m.as<u64>());
        if (rc) return rc;
        FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    }
    return FHEON_OK;
}

int decode_dev(fheon_ctx *ctx, const fheon_pt *pt, double *re, double *im, u32 nz)
{
    const u32 N = ctx->N, n = N / 2, nl = pt->level >= 2 ? 2 : 1;
    cudaStream_t st = ctx->stream;
    DevMem c, U, V, zo;
    if (!c.alloc((size_t)nl * N * 8, st) || !U.alloc((size_t)n * 16, st) || !V.alloc((size_t)n * 16, st) ||
        !zo.alloc((size_t)2 * n * 8, st))
        return fail(ctx, FHEON_ERR_OOM, "decode temporaries");
    FHEON_CUDA(ctx, ntt_inv_limbs(ctx, pt->m.as<u64>(), c.as<u64>(), nl, ctx->L, 0, st));
    const u64 q0 = ctx->mod[0], q1 = nl == 2 ? ctx->mod[1] : 1;
    const u64 inv = nl == 2 ? h_invmod(q0 % q1, q1) : 0;
    decode_lift_kernel<<<nblk(n), TPB, 0, st>>>(c.as<u64>(), nl, q0, q1, inv, nl == 2 ? h_shoup(inv, q1) : 0,
                                                ctx->tab.fft_zeta.as<double2>(), U.as<double2>(), n, 1.0 / pt->scale);
    FHEON_CUDA(ctx, fft(ctx, U.as<double2>(), V.as<double2>(), +1));
    double *dre = zo.as<double>(), *dim = dre + n;
    slot_gather_kernel<<<nblk(nz), TPB, 0, st>>>(V.as<double2>(), ctx->tab.slot_perm.as<u32>(), dre, dim, nz);
    FHEON_CUDA(ctx, cudaGetLastError());
    FHEON_CUDA(ctx, cudaMemcpyAsync(re, dre, (size_t)nz * 8, cudaMemcpyDeviceToHost, st));
    if (im) FHEON_CUDA(ctx, cudaMemcpyAsync(im, dim, (size_t)nz * 8, cudaMemcpyDeviceToHost, st));
    FHEON_CUDA(ctx, cudaStreamSynchronize(st));
    return FHEON_OK;
}

} // namespace fheon
