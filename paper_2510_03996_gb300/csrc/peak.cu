// peak.cu -- measured rates of the modular steps the ALU-bound kernels are
// built from, the denominators of their rooflines.
//
// The NTT passes and the fused base conversions of the rotation path are
// bound by integer issue, not by HBM, and the GPU has no published 64-bit
// modular-multiply rate.  Each kernel below runs one of those steps alone,
// in the form and with the operands the production kernels use, on every SM
// at the occupancy those kernels run at:
//   FHEON_PEAK_CT_LAZY   forward (Cooley-Tukey) butterfly without conditional
//                        subtractions (primes below 2^54);
//   FHEON_PEAK_GS_LAZY   inverse (Gentleman-Sande) butterfly, same primes;
//   FHEON_PEAK_CT_HARVEY forward butterfly with Harvey's reductions (any
//                        prime below 2^62);
//   FHEON_PEAK_GS_HARVEY inverse butterfly with Harvey's reductions;
//   FHEON_PEAK_MAC       128-bit multiply-accumulate of a base conversion
//                        (one source word times a Montgomery constant).
// Each step is timed at two occupancies (2 and 3 resident 256-thread CTAs per
// SM) and the faster counts.  A butterfly thread holds 16 words and runs radix-16 rounds of four stages
// (32 butterflies, 15 twiddle pairs read through the read-only cache per
// round), as a round of ntt_core.cuh does; its shared-memory exchange is left
// out, so the rate is that of the arithmetic alone.  A conversion thread
// reads four source words per round and multiplies each into eight
// accumulators, as the fused conversions do, reducing each accumulator once
// per round.
#include <algorithm>

#include "internal.h"
#include "ntt_core.cuh"

using namespace fheon;

namespace {

constexpr int PEAK_THREADS = 256;
constexpr u32 TW_ENTRIES = 256;

// BPS: resident CTAs per SM the registers are sized for (2: up to 128
// registers a thread, 3: up to 85, as the production passes)
template <int KIND, int BPS>
__global__ void __launch_bounds__(PEAK_THREADS, BPS)
    peak_kernel(const ulonglong2 *__restrict__ tw, const u64 *__restrict__ src, ModConst mc, u32 rounds, u64 *out)
{
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q = mc.q, twoq = mc.twoq;
    u64 fold = 0;
    if constexpr (KIND == FHEON_PEAK_MAC) {
        u64 cst[8];
#pragma unroll
        for (int j = 0; j < 8; j++) cst[j] = tw[(t + j) & (TW_ENTRIES - 1)].x;
        for (u32 rd = 0; rd < rounds; rd++) {
            u128acc a[8];
#pragma unroll
            for (int j = 0; j < 8; j++) acc_zero(a[j]);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const u64 x = __ldg(&src[(t + rd * 4 + i) & (TW_ENTRIES - 1)]);
#pragma unroll
                for (int j = 0; j < 8; j++) acc_mad(a[j], x, cst[j]);
            }
#pragma unroll
            for (int j = 0; j < 8; j++) fold ^= redc_lazy(a[j].hi, a[j].lo, q, mc.qneg_inv);
        }
    } else {
        u64 x[16];
#pragma unroll
        for (int v = 0; v < 16; v++) x[v] = (u64)t * 16 + v;
        for (u32 rd = 0; rd < rounds; rd++) {
            const u32 base = (rd * 15 + t) & (TW_ENTRIES - 1);
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const int vb = (KIND == FHEON_PEAK_GS_LAZY || KIND == FHEON_PEAK_GS_HARVEY) ? s : 3 - s;
                const u64 cst = twoq << s;
#pragma unroll
                for (int v = 0; v < 16; v++) {
                    if ((v >> vb) & 1) continue;
                    // one twiddle per butterfly group of the stage: 1, 2, 4, 8 per stage
                    const int grp = v >> (vb + 1);
                    const ulonglong2 w = __ldg(&tw[(base + (1 << (3 - vb)) - 1 + grp) & (TW_ENTRIES - 1)]);
                    u64 &X = x[v], &Y = x[v | (1 << vb)];
                    if constexpr (KIND == FHEON_PEAK_CT_LAZY) {
                        const u64 tt = shoup_lazy(Y, w.x, w.y, q);
                        Y = X - tt + twoq;
                        X = X + tt;
                    } else if constexpr (KIND == FHEON_PEAK_GS_LAZY) {
                        const u64 d = X - Y + cst;
                        X = X + Y;
                        Y = shoup_lazy(d, w.x, w.y, q);
                    } else if constexpr (KIND == FHEON_PEAK_CT_HARVEY) {
                        ct_butterfly(X, Y, w.x, w.y, q, twoq);
                    } else {
                        gs_butterfly(X, Y, w.x, w.y, q, twoq);
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < 16; v++) fold ^= x[v];
    }
    // the result is kept so that no step can be removed; one word per thread
    out[t] = fold;
}

template <int KIND>
cudaError_t launch_peak(u32 bps, u32 sms, const ulonglong2 *tw, const u64 *src, const ModConst &mc, u32 rounds,
                        u64 *out, cudaStream_t st)
{
    if (bps == 2) peak_kernel<KIND, 2><<<sms * 2, PEAK_THREADS, 0, st>>>(tw, src, mc, rounds, out);
    else peak_kernel<KIND, 3><<<sms * 3, PEAK_THREADS, 0, st>>>(tw, src, mc, rounds, out);
    return cudaGetLastError();
}

cudaError_t launch_kind(u32 kind, u32 bps, u32 sms, const ulonglong2 *tw, const u64 *src, const ModConst &mc,
                        u32 rounds, u64 *out, cudaStream_t st)
{
    switch (kind) {
    case FHEON_PEAK_CT_LAZY: return launch_peak<FHEON_PEAK_CT_LAZY>(bps, sms, tw, src, mc, rounds, out, st);
    case FHEON_PEAK_GS_LAZY: return launch_peak<FHEON_PEAK_GS_LAZY>(bps, sms, tw, src, mc, rounds, out, st);
    case FHEON_PEAK_CT_HARVEY: return launch_peak<FHEON_PEAK_CT_HARVEY>(bps, sms, tw, src, mc, rounds, out, st);
    case FHEON_PEAK_GS_HARVEY: return launch_peak<FHEON_PEAK_GS_HARVEY>(bps, sms, tw, src, mc, rounds, out, st);
    case FHEON_PEAK_MAC: return launch_peak<FHEON_PEAK_MAC>(bps, sms, tw, src, mc, rounds, out, st);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace

extern "C" int fheon_alu_peak(fheon_ctx *ctx, uint32_t kind, uint32_t rounds, uint32_t reps, double *per_s)
{
    if (!ctx || !per_s || kind >= FHEON_PEAK_KINDS || rounds == 0 || rounds > (1u << 20) || reps == 0 || reps > 100)
        return FHEON_ERR_ARG;
    // the prime class the step is used with: lazy butterflies only below 2^54
    const bool lazy = kind == FHEON_PEAK_CT_LAZY || kind == FHEON_PEAK_GS_LAZY;
    int mi = -1;
    for (u32 i = 0; i < ctx->L + ctx->K && mi < 0; i++)
        if (!lazy || ctx->mod[i] < ntt::LAZY_BOUND) mi = (int)i;
    if (mi < 0) return fail(ctx, FHEON_ERR_ARG, "alu peak: no prime below 2^54 for a lazy butterfly");
    int dev = 0, sms = 0;
    FHEON_CUDA(ctx, cudaGetDevice(&dev));
    FHEON_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (ctx->N < TW_ENTRIES) return fail(ctx, FHEON_ERR_ARG, "alu peak: N below %u", TW_ENTRIES);
    const size_t max_threads = (size_t)sms * 3 * PEAK_THREADS;
    DevMem out, src;
    if (!out.alloc(max_threads * 8, ctx->stream) || !src.alloc(TW_ENTRIES * 8, ctx->stream))
        return fail(ctx, FHEON_ERR_OOM, "alu peak: device memory");
    // twiddles: the context's own forward table of that prime; sources: its residues
    const ulonglong2 *tw = ctx->tab.tw_fwd.as<ulonglong2>() + (size_t)mi * ctx->N;
    FHEON_CUDA(ctx, cudaMemcpy2DAsync(src.p, 8, tw, 16, 8, TW_ENTRIES, cudaMemcpyDeviceToDevice, ctx->stream));
    const ModConst mc = ctx->mc[mi];
    cudaEvent_t e0, e1;
    FHEON_CUDA(ctx, cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ctx, e, "cudaEventCreate");
    }
    // the faster of two occupancies: 2 CTAs per SM (no register limit short of
    // 128) and 3 (the production passes' budget)
    double best_rate = 0.0;
    for (u32 bps = 2; bps <= 3 && e == cudaSuccess; bps++) {
        const double threads = (double)sms * bps * PEAK_THREADS;
        e = launch_kind(kind, bps, (u32)sms, tw, src.as<u64>(), mc, rounds, out.as<u64>(), ctx->stream); // warm-up
        for (u32 r = 0; r < reps && e == cudaSuccess; r++) {
            if ((e = cudaEventRecord(e0, ctx->stream)) != cudaSuccess) break;
            if ((e = launch_kind(kind, bps, (u32)sms, tw, src.as<u64>(), mc, rounds, out.as<u64>(), ctx->stream)) !=
                cudaSuccess)
                break;
            if ((e = cudaEventRecord(e1, ctx->stream)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.0f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
            // 32 butterflies (four stages of eight) or 32 multiply-accumulates
            // (four sources times eight accumulators) per round and thread
            if (ms > 0.0f) best_rate = std::max(best_rate, threads * rounds * 32.0 / (ms / 1e3));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "alu peak");
    *per_s = best_rate;
    return FHEON_OK;
}
