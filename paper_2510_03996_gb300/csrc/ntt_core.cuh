// ntt_core.cuh -- batched 64-bit negacyclic NTT / INTT for sm_103a.
//
// Transform (the convention every kernel and the key material share): for a
// limb a over prime q with smallest primitive 2N-th root psi, the forward
// transform writes out[j] = a(psi^(2*brv(j)+1)), i.e. the Cooley-Tukey
// "merged" negacyclic NTT with bit-reversed output (Longa-Naehrig 2016); the
// inverse is the Gentleman-Sande transform back to natural order times N^-1
// (times an optional per-limb constant folded into the last multiply).
//
// A butterfly at half-size t = 2^tau on lower index J uses twiddle number
// 2^(logN-1-tau) + (J >> (tau+1)) of the table psi^brv(i) (forward) or
// psi^-brv(i) (inverse); tables hold (w, floor(w*2^64/q)) pairs.
//
// GB300 mapping.  One limb of N = 2^16 u64 is 512 KiB, more than a CTA's
// shared memory, so each transform is two passes over a limb viewed as an
// N1 x N2 matrix (J = u*N2 + c):
//   pass A ("columns"): the butterflies on the high log2(N1) bits of J; a CTA
//     owns SUBS adjacent columns, so warps read 128-byte row segments;
//   pass B ("rows"):    the butterflies on the low log2(N2) bits; a CTA owns
//     SUBS contiguous rows.
// Forward runs A then B, inverse B then A; the second pass works in place on
// the first pass's output (intermediate values stay lazily reduced).  Inside
// a pass each thread keeps R = 16 elements in registers and does 4 stages per
// round (radix 16), exchanging through shared memory between rounds; the
// row layout is padded by one word per 16 so strided rounds are free of bank
// conflicts.  Loads and stores of the tile go through a Job policy, which is
// where automorphism gathers, base conversions and epilogues fuse in.
#pragma once
#include <cuda_runtime.h>

#include "modarith.cuh"

namespace fheon {
// Instrumentation hook: records a CUDA event named `name` on `st` after the
// preceding launch when the calling thread's context is being profiled.
void prof_mark(cudaStream_t st, const char *name);
}

namespace ntt {

constexpr int LOGR = 4;
constexpr int R = 1 << LOGR;
constexpr int TILE_ELEMS = 4096;
constexpr int NTHREADS = 256;

template <int LOGN>
struct Cfg {
    static constexpr int B1 = LOGN / 2;      // pass A bits (high)
    static constexpr int B2 = LOGN - B1;     // pass B bits (low)
    static constexpr int N1 = 1 << B1, N2 = 1 << B2;
    static constexpr int TILE = (1 << LOGN) < TILE_ELEMS ? (1 << LOGN) : TILE_ELEMS;
    static constexpr int ROW_SUBS = TILE / N2;                          // rows per CTA (pass B)
    static constexpr int COL_SUBS = (TILE / N1) < N2 ? (TILE / N1) : N2; // columns per CTA (pass A)
    static constexpr int ROW_THREADS = ROW_SUBS * (N2 / R);
    static constexpr int COL_THREADS = COL_SUBS * (N1 / R);
    static constexpr int ROW_TILES = N1 / ROW_SUBS;
    static constexpr int COL_TILES = N2 / COL_SUBS;
    static constexpr int ROW_SMEM = ROW_SUBS * (N2 + N2 / 16) * 8;
    static constexpr int COL_SMEM = COL_SUBS * N1 * 8;
};

// One pass.  ROWS: pass B, else pass A.  FIRST: this is the first of the two
// passes (loads through Job::load_first, stores raw to Job::mid), else the
// second (loads Job::mid, stores through Job::store_last).
template <int LOGN, bool INV, bool ROWS, bool FIRST, class Job>
__global__ void __launch_bounds__(256) pass_kernel(const __grid_constant__ typename Job::Params prm)
{
    using C = Cfg<LOGN>;
    constexpr int LOGM = ROWS ? C::B2 : C::B1;
    constexpr int M = 1 << LOGM;
    constexpr int G = M / R;                       // threads per sub-transform
    constexpr int SUBS = ROWS ? C::ROW_SUBS : C::COL_SUBS;
    constexpr int NT = SUBS * G;
    constexpr int TILES = ROWS ? C::ROW_TILES : C::COL_TILES;
    constexpr int ROUNDS = (LOGM + LOGR - 1) / LOGR;
    constexpr int RSTRIDE = M + M / 16;

    extern __shared__ u64 sm[];
    const u32 job_i = blockIdx.x / TILES;
    const u32 tile = blockIdx.x % TILES;
    Job job(prm, job_i);
    if (!job.active()) return;
    const ModConst mc = job.mod();
    const ulonglong2 *__restrict__ tw = job.twiddles(INV);
    const u64 q = mc.q, twoq = mc.twoq;
    const int t = threadIdx.x;

    // ---- load the tile (coalesced) ----
#pragma unroll
    for (int k = 0; k < R; k++) {
        const int lin = t + k * NT;
        int sub, e;
        if (ROWS) { sub = lin / M; e = lin % M; }
        else { sub = lin % SUBS; e = lin / SUBS; }
        const u32 J = ROWS ? (u32)((tile * SUBS + sub) * M + e) : (u32)(e * C::N2 + tile * SUBS + sub);
        const int s = ROWS ? sub * RSTRIDE + e + (e >> 4) : e * SUBS + sub;
        sm[s] = FIRST ? job.template load_first<INV>(J) : job.load_mid(J);
    }
    __syncthreads();

    int sub, g;
    if (ROWS) { sub = t / G; g = t % G; }
    else { sub = t % SUBS; g = t / SUBS; }
    const u32 row = (u32)(tile * SUBS + sub); // global row (pass B only)

    u64 x[R];
#pragma unroll
    for (int rd = 0; rd < ROUNDS; rd++) {
        const int lo = INV ? rd * LOGR : ((LOGM - (rd + 1) * LOGR) > 0 ? LOGM - (rd + 1) * LOGR : 0);
        const int nb = INV ? ((LOGM - lo) < LOGR ? LOGM - lo : LOGR) : (LOGM - rd * LOGR) - lo;
        int e[R];
#pragma unroll
        for (int v = 0; v < R; v++) {
            const int rest = (g << (LOGR - nb)) | (v >> nb);
            const int lowp = rest & ((1 << lo) - 1);
            const int highp = rest >> lo;
            e[v] = (highp << (lo + nb)) | ((v & ((1 << nb) - 1)) << lo) | lowp;
            x[v] = sm[ROWS ? sub * RSTRIDE + e[v] + (e[v] >> 4) : e[v] * SUBS + sub];
        }
#pragma unroll
        for (int s = 0; s < nb; s++) {
            const int vb = INV ? s : nb - 1 - s;
            const int b = lo + vb;                       // local bit of this stage
            const int tau = b + (ROWS ? 0 : C::B2);      // global bit
            ulonglong2 w = make_ulonglong2(0, 0);
#pragma unroll
            for (int v = 0; v < R; v++) {
                if ((v >> vb) & 1) continue;
                if ((v & ((1 << vb) - 1)) == 0) {
                    const u32 prefix = ROWS ? ((row << (LOGM - 1 - b)) + ((u32)e[v] >> (b + 1)))
                                            : ((u32)e[v] >> (b + 1));
                    w = __ldg(&tw[(1u << (LOGN - 1 - tau)) + prefix]);
                }
                if (INV) gs_butterfly(x[v], x[v | (1 << vb)], w.x, w.y, q, twoq);
                else ct_butterfly(x[v], x[v | (1 << vb)], w.x, w.y, q, twoq);
            }
        }
#pragma unroll
        for (int v = 0; v < R; v++) sm[ROWS ? sub * RSTRIDE + e[v] + (e[v] >> 4) : e[v] * SUBS + sub] = x[v];
        __syncthreads();
    }

    // ---- store the tile (coalesced) ----
#pragma unroll
    for (int k = 0; k < R; k++) {
        const int lin = t + k * NT;
        int sb, e;
        if (ROWS) { sb = lin / M; e = lin % M; }
        else { sb = lin % SUBS; e = lin / SUBS; }
        const u32 J = ROWS ? (u32)((tile * SUBS + sb) * M + e) : (u32)(e * C::N2 + tile * SUBS + sb);
        const u64 val = sm[ROWS ? sb * RSTRIDE + e + (e >> 4) : e * SUBS + sb];
        if (FIRST) job.store_mid(J, val);
        else job.template store_last<INV>(J, val, mc);
    }
}

// Launch both passes of a forward (INV = false) or inverse transform over
// `njobs` limbs described by Job.
template <int LOGN, bool INV, class Job>
inline cudaError_t launch_fixed(const typename Job::Params &prm, u32 njobs, cudaStream_t st)
{
    using C = Cfg<LOGN>;
    if (njobs == 0) return cudaSuccess;
    constexpr bool FIRST_ROWS = INV; // inverse starts with rows, forward with columns
    auto k1 = pass_kernel<LOGN, INV, FIRST_ROWS, true, Job>;
    auto k2 = pass_kernel<LOGN, INV, !FIRST_ROWS, false, Job>;
    const int th1 = FIRST_ROWS ? C::ROW_THREADS : C::COL_THREADS;
    const int th2 = FIRST_ROWS ? C::COL_THREADS : C::ROW_THREADS;
    const int sm1 = FIRST_ROWS ? C::ROW_SMEM : C::COL_SMEM;
    const int sm2 = FIRST_ROWS ? C::COL_SMEM : C::ROW_SMEM;
    const int tl1 = FIRST_ROWS ? C::ROW_TILES : C::COL_TILES;
    const int tl2 = FIRST_ROWS ? C::COL_TILES : C::ROW_TILES;
    static_assert(C::ROW_SMEM <= 48 * 1024 && C::COL_SMEM <= 48 * 1024, "tile exceeds default shared memory");
    k1<<<dim3(njobs * tl1), dim3(th1), sm1, st>>>(prm);
    fheon::prof_mark(st, INV ? "ntt_inv_rows" : "ntt_fwd_cols");
    k2<<<dim3(njobs * tl2), dim3(th2), sm2, st>>>(prm);
    fheon::prof_mark(st, INV ? "ntt_inv_cols" : "ntt_fwd_rows");
    return cudaGetLastError();
}

template <bool INV, class Job>
inline cudaError_t launch(u32 logN, const typename Job::Params &prm, u32 njobs, cudaStream_t st)
{
    switch (logN) {
    case 10: return launch_fixed<10, INV, Job>(prm, njobs, st);
    case 11: return launch_fixed<11, INV, Job>(prm, njobs, st);
    case 12: return launch_fixed<12, INV, Job>(prm, njobs, st);
    case 13: return launch_fixed<13, INV, Job>(prm, njobs, st);
    case 14: return launch_fixed<14, INV, Job>(prm, njobs, st);
    case 15: return launch_fixed<15, INV, Job>(prm, njobs, st);
    case 16: return launch_fixed<16, INV, Job>(prm, njobs, st);
    case 17: return launch_fixed<17, INV, Job>(prm, njobs, st);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace ntt
