// ntt_core.cuh -- batched 64-bit negacyclic NTT / INTT for sm_103a.
//
// Transform (the convention every kernel and the key material share): for a
// limb a over prime q with smallest primitive 2N-th root psi, the forward
// transform writes out[j] = a(psi^(2*brv(j)+1)), i.e. the Cooley-Tukey
// "merged" negacyclic NTT with bit-reversed output (Longa-Naehrig 2016); the
// inverse is the Gentleman-Sande transform back to natural order times N^-1
// (times an optional per-limb constant folded into that last multiply).
//
// A butterfly at half-size t = 2^tau on lower index J uses twiddle number
// 2^(logN-1-tau) + (J >> (tau+1)) of the table psi^brv(i) (forward) or
// psi^-brv(i) (inverse); tables hold (w, floor(w*2^64/q)) pairs.
//
// GB300 mapping.  One limb of N = 2^16 u64 is 512 KiB, more than a CTA's
// shared memory, so each transform is two passes over a limb viewed as an
// N1 x N2 matrix (J = u*N2 + c):
//   pass A ("columns"): butterflies on the high log2(N1) bits of J; a CTA owns
//     SUBS adjacent columns, so a warp touches 128-byte row segments;
//   pass B ("rows"):    butterflies on the low log2(N2) bits; a CTA owns SUBS
//     contiguous rows.
// Forward runs A then B, inverse B then A; the second pass reads the first
// pass's output (lazily reduced) from the job's mid buffer.  Each thread keeps
// R = 16 elements in registers and does 4 stages per round (radix 16),
// exchanging through shared memory between rounds (rows padded by one word
// per 16: no bank conflicts).  Where a round's register layout is already
// coalesced in global memory (forward loads, most stores), the tile moves
// straight between registers and global memory; elsewhere it is staged
// through shared memory.
//
// Reduction.  For primes below 2^54 the butterflies skip every conditional
// subtraction: forward outputs stay below x_in + 2q (at most 35q after 17
// stages), inverse values below 2^(s+1) q at stage s of a pass with the
// stage constant 2^(s+1) q keeping X - Y + C non-negative; one Shoup-by-one
// reduction at the second pass's load and at the end makes them canonical.
// Larger primes use Harvey's lazy butterflies ([0, 4q) forward, [0, 2q)
// inverse).
//
// Jobs.  Loads, stores, the limb's modulus and twiddles come from a Job
// policy.  A job may also repeat the transform over several inputs that
// share one output (`reps`; the key inner product sums digits this way), pass
// an input through without transforming it, and finish with a per-element
// epilogue.
#pragma once
#include <cuda_runtime.h>

#include "modarith.cuh"

namespace fheon {
// Instrumentation hook: records a CUDA event named `name` on `st` after the
// preceding launch while a profile is open on that stream.
void prof_mark(cudaStream_t st, const char *name);
} // namespace fheon

namespace ntt {

constexpr int LOGR = 4; // radix of the column passes, and the default of the row passes
constexpr int R = 1 << LOGR;
constexpr int TILE_ELEMS = 4096;
constexpr u64 LAZY_BOUND = 1ull << 54;

// LOGR_ROWS: radix of the row passes (4: radix 16, 4096-element tiles; 3:
// radix 8, 2048-element tiles, still 256 threads a CTA and half the registers
// a thread).  The column passes are radix 16 either way: a radix-8 column
// tile would read 64-byte instead of 128-byte row segments.
template <int LOGN, int LOGR_ROWS = LOGR>
struct Cfg {
    static constexpr int B1 = LOGN / 2;  // pass A bits (high)
    static constexpr int B2 = LOGN - B1; // pass B bits (low)
    static constexpr int N1 = 1 << B1, N2 = 1 << B2;
    static constexpr int RR = 1 << LOGR_ROWS;
    static constexpr int TILE = (1 << LOGN) < TILE_ELEMS ? (1 << LOGN) : TILE_ELEMS;
    static constexpr int ROW_TILE_ELEMS = 256 * RR;
    static constexpr int ROW_TILE = (1 << LOGN) < ROW_TILE_ELEMS ? (1 << LOGN) : ROW_TILE_ELEMS;
    static constexpr int ROW_SUBS = ROW_TILE / N2;                       // rows per CTA (pass B)
    static constexpr int COL_SUBS = (TILE / N1) < N2 ? (TILE / N1) : N2; // columns per CTA (pass A)
    static constexpr int ROW_THREADS = ROW_SUBS * (N2 / RR);
    static constexpr int COL_THREADS = COL_SUBS * (N1 / R);
    static constexpr int ROW_TILES = N1 / ROW_SUBS;
    static constexpr int COL_TILES = N2 / COL_SUBS;
    static constexpr int ROW_SMEM = ROW_SUBS * (N2 + N2 / 16) * 8;
    static constexpr int COL_SMEM = COL_SUBS * N1 * 8;
};

// Defaults for the optional parts of the Job interface.
struct JobBase {
    // resident 256-thread CTAs per SM the register budget is sized for: 3 for
    // plain transforms (<= 85 registers, no spills), 2 for jobs with fused
    // base conversions or accumulations
    static constexpr int MIN_BLOCKS = 3;
    // extra shared memory the job needs, in u64 words per tile element; the
    // kernel hands it over with attach()
    static constexpr int EXTRA_WORDS_PER_ELEM = 0;
    // true when the extra size depends on the launch parameters: the job then
    // provides  static __host__ __device__ u32 extra_words(const Params &)
    static constexpr bool RUNTIME_EXTRA = false;
    __device__ void attach(u64 *) {}
    __device__ int reps() const { return 1; }
    // start of repetition `rep` on tile `tile` of `te` consecutive elements of
    // the pass's grid (jobs prefetch their operands here)
    __device__ void begin(int, u32, u32) {}
    __device__ bool passthrough() const { return false; }
    __device__ u64 load_passthrough(u32) const { return 0; }
    __device__ void finish(int, u32, const ModConst &) {}
    // whole-tile direct loads of the first pass (default: element by element)
    static constexpr bool TILE_LOAD = false;
    // whole-tile stores of the second pass: store_tile_last(J[RR], value[RR],
    // mod) gets every final value of the thread at once (RR: the pass's radix),
    // so a job that reads operands to combine with them can issue those loads
    // together
    static constexpr bool TILE_STORE = false;
    // a forward transform over a lazy prime may hand its consumer the values
    // unreduced (below 36q for up to 17 stages from inputs below 2q)
    static constexpr bool LAZY_OUT = false;
    // a first row pass whose input is a Galois image sigma_g(in): the job gives
    // gather_src(J) (the input index element J reads) and gather_dst(s) (its
    // inverse) and load_src(s) = in[s]; the tile's sources are one aligned
    // tile of `in`, read in order (coalesced) and placed in shared memory at
    // their destinations
    static constexpr bool GATHER_LOAD = false;
};

// reduce v < 2^64 to [0, q) with one Shoup product by 1 and a subtraction
__device__ __forceinline__ u64 reduce_any(u64 v, const ModConst &m)
{
    u64 r = v - __umul64hi(v, m.one_sh) * m.q;
    return r >= m.q ? r - m.q : r;
}
__device__ __forceinline__ u64 reduce_any_lazy(u64 v, const ModConst &m) { return v - __umul64hi(v, m.one_sh) * m.q; }

template <int LOGN, bool INV, bool ROWS, bool FIRST, bool LAZY, class Job, int LOGR_ROWS = LOGR>
__device__ __forceinline__ void pass_body(Job &job, u32 tile)
{
    using C = Cfg<LOGN, LOGR_ROWS>;
    constexpr int LOGR = ROWS ? LOGR_ROWS : ntt::LOGR; // this pass's radix
    constexpr int R = 1 << LOGR;
    constexpr int LOGM = ROWS ? C::B2 : C::B1;
    constexpr int M = 1 << LOGM;
    constexpr int G = M / R;
    constexpr int SUBS = ROWS ? C::ROW_SUBS : C::COL_SUBS;
    constexpr int NT = SUBS * G;
    constexpr int ROUNDS = (LOGM + LOGR - 1) / LOGR;
    constexpr int RSTRIDE = M + M / 16;
    // round 0 of a forward pass covers the top bits: e = v*G + g, coalesced in
    // both passes; an inverse column pass starts on the low bits of u, which
    // are still coalesced across its lanes (lanes differ in the column).
    constexpr bool DIRECT_LOAD = !INV || !ROWS;
    // the last round of a forward row pass covers the low bits: a thread owns
    // 16 consecutive words, so that store is staged; every other last round is
    // coalesced across lanes.
    constexpr bool DIRECT_STORE = INV || !ROWS;

    extern __shared__ u64 sm[];
    job.attach(sm + (ROWS ? SUBS * RSTRIDE : SUBS * M));
    const int t = threadIdx.x;
    int sub, g;
    if (ROWS) { sub = t / G; g = t % G; }
    else { sub = t % SUBS; g = t / SUBS; }
    const u32 line = (u32)(tile * SUBS + sub); // global row (pass B) or column (pass A)

    auto gidx = [&](int sb, int e) -> u32 {
        return ROWS ? (u32)((tile * SUBS + sb) * M + e) : (u32)(e * C::N2 + tile * SUBS + sb);
    };
    auto sidx = [&](int sb, int e) -> int { return ROWS ? sb * RSTRIDE + e + (e >> 4) : e * SUBS + sb; };
    // element of register v in round rd
    auto relem = [&](int rd, int v) -> int {
        const int lo = INV ? rd * LOGR : ((LOGM - (rd + 1) * LOGR) > 0 ? LOGM - (rd + 1) * LOGR : 0);
        const int nb = INV ? ((LOGM - lo) < LOGR ? LOGM - lo : LOGR) : (LOGM - rd * LOGR) - lo;
        const int rest = (g << (LOGR - nb)) | (v >> nb);
        return ((rest >> lo) << (lo + nb)) | ((v & ((1 << nb) - 1)) << lo) | (rest & ((1 << lo) - 1));
    };
    // element index of store slot k (register v in the last round, or the staged linear slot)
    auto store_J = [&](int k) -> u32 {
        if (DIRECT_STORE) return gidx(sub, relem(ROUNDS - 1, k));
        const int lin = t + k * NT;
        return ROWS ? gidx(lin / M, lin % M) : gidx(lin % SUBS, lin / SUBS);
    };

    const int nrep = job.reps();
    for (int rep = 0; rep < nrep; rep++) {
        job.begin(rep, tile, (u32)(SUBS * M));
        // the modulus may change between repetitions (a job may run one
        // transform per target limb over shared sources)
        const ModConst mc = job.mod();
        const ulonglong2 *__restrict__ tw = job.twiddles(INV);
        const u64 q = mc.q, twoq = mc.twoq;
        if (job.passthrough()) {
#pragma unroll
            for (int k = 0; k < R; k++) {
                const u32 J = store_J(k);
                job.store_last(k, J, job.load_passthrough(J), mc);
            }
            continue;
        }
        u64 x[R];
        // ---- load ----
        if constexpr (DIRECT_LOAD && FIRST && Job::TILE_LOAD) {
            u32 Js[R];
            int Ss[R];
#pragma unroll
            for (int v = 0; v < R; v++) {
                Js[v] = gidx(sub, relem(0, v));
                Ss[v] = sidx(sub, relem(0, v));
            }
            job.load_tile_first(Js, Ss, x);
        } else if (DIRECT_LOAD) {
#pragma unroll
            for (int v = 0; v < R; v++) {
                const u32 J = gidx(sub, relem(0, v));
                x[v] = FIRST ? job.template load_first<INV>(J) : job.load_mid(J);
            }
        } else if constexpr (FIRST && Job::GATHER_LOAD) {
            static_assert(ROWS, "a gathered load needs the row pass: a tile of consecutive elements");
            const u32 t0 = tile * (u32)(SUBS * M);
            const u32 s0 = job.gather_src(t0) & ~(u32)(SUBS * M - 1);
            u64 v_[R];
#pragma unroll
            for (int k = 0; k < R; k++) v_[k] = job.load_src(s0 + (u32)(t + k * NT));
#pragma unroll
            for (int k = 0; k < R; k++) {
                const u32 loc = job.gather_dst(s0 + (u32)(t + k * NT)) - t0;
                sm[sidx((int)(loc / M), (int)(loc % M))] = v_[k];
            }
            __syncthreads();
#pragma unroll
            for (int v = 0; v < R; v++) x[v] = sm[sidx(sub, relem(0, v))];
        } else {
#pragma unroll
            for (int k = 0; k < R; k++) {
                const int lin = t + k * NT;
                const int sb = ROWS ? lin / M : lin % SUBS, e = ROWS ? lin % M : lin / SUBS;
                const u32 J = gidx(sb, e);
                sm[sidx(sb, e)] = FIRST ? job.template load_first<INV>(J) : job.load_mid(J);
            }
            __syncthreads();
#pragma unroll
            for (int v = 0; v < R; v++) x[v] = sm[sidx(sub, relem(0, v))];
        }
        if (LAZY && INV && !FIRST) {
#pragma unroll
            for (int v = 0; v < R; v++) x[v] = reduce_any_lazy(x[v], mc); // < 2q
        }
        // ---- rounds ----
#pragma unroll
        for (int rd = 0; rd < ROUNDS; rd++) {
            const int lo = INV ? rd * LOGR : ((LOGM - (rd + 1) * LOGR) > 0 ? LOGM - (rd + 1) * LOGR : 0);
            const int nb = INV ? ((LOGM - lo) < LOGR ? LOGM - lo : LOGR) : (LOGM - rd * LOGR) - lo;
            if (rd > 0) {
#pragma unroll
                for (int v = 0; v < R; v++) x[v] = sm[sidx(sub, relem(rd, v))];
            }
#pragma unroll
            for (int s = 0; s < nb; s++) {
                const int vb = INV ? s : nb - 1 - s;
                const int b = lo + vb;                  // local bit of this stage
                const int tau = b + (ROWS ? 0 : C::B2); // global bit
                const int sp = INV ? rd * LOGR + s : 0; // stage index within an inverse pass
                const u64 cst = twoq << sp;             // 2^(sp+1) q: keeps X - Y + C >= 0 (lazy inverse)
                ulonglong2 w = make_ulonglong2(0, 0);
#pragma unroll
                for (int v = 0; v < R; v++) {
                    if ((v >> vb) & 1) continue;
                    const int e = relem(rd, v);
                    if ((v & ((1 << vb) - 1)) == 0) {
                        const u32 prefix = ROWS ? ((line << (LOGM - 1 - b)) + ((u32)e >> (b + 1))) : ((u32)e >> (b + 1));
                        w = __ldg(&tw[(1u << (LOGN - 1 - tau)) + prefix]);
                    }
                    u64 &X = x[v], &Y = x[v | (1 << vb)];
                    if (INV) {
                        if (LAZY) {
                            const u64 d = X - Y + cst;
                            X = X + Y;
                            Y = shoup_lazy(d, w.x, w.y, q);
                        } else {
                            gs_butterfly(X, Y, w.x, w.y, q, twoq);
                        }
                    } else {
                        if (LAZY) {
                            const u64 tt = shoup_lazy(Y, w.x, w.y, q);
                            Y = X - tt + twoq;
                            X = X + tt;
                        } else {
                            ct_butterfly(X, Y, w.x, w.y, q, twoq);
                        }
                    }
                }
            }
            if (rd < ROUNDS - 1) {
#pragma unroll
                for (int v = 0; v < R; v++) sm[sidx(sub, relem(rd, v))] = x[v];
                __syncthreads();
            }
        }
        // ---- store ----
        auto final_value = [&](u64 val) -> u64 {
            if (INV) {
                const ulonglong2 s = job.inv_scale();
                return shoup(val, s.x, s.y, q); // any input < 2^64
            }
            if (LAZY && Job::LAZY_OUT) return val;
            return LAZY ? reduce_any(val, mc) : reduce4q(val, q);
        };
        auto emit = [&](int k, u32 J, u64 val) {
            if (FIRST) job.store_mid(J, val);
            else job.store_last(k, J, final_value(val), mc);
        };
        if (!DIRECT_STORE) {
#pragma unroll
            for (int v = 0; v < R; v++) sm[sidx(sub, relem(ROUNDS - 1, v))] = x[v];
            __syncthreads();
        }
        // element and value of store slot k
        auto slot = [&](int k, u32 &J, u64 &val) {
            if (DIRECT_STORE) {
                J = gidx(sub, relem(ROUNDS - 1, k));
                val = x[k];
            } else {
                const int lin = t + k * NT;
                const int sb = ROWS ? lin / M : lin % SUBS, e = ROWS ? lin % M : lin / SUBS;
                J = gidx(sb, e);
                val = sm[sidx(sb, e)];
            }
        };
        if constexpr (!FIRST && Job::TILE_STORE) {
            u32 Js[R];
            u64 vs[R];
#pragma unroll
            for (int k = 0; k < R; k++) {
                slot(k, Js[k], vs[k]);
                vs[k] = final_value(vs[k]);
            }
            job.store_tile_last(Js, vs, mc);
        } else {
#pragma unroll
            for (int k = 0; k < R; k++) {
                u32 J;
                u64 val;
                slot(k, J, val);
                emit(k, J, val);
            }
        }
        if (nrep > 1) __syncthreads(); // the next repetition reuses shared memory
    }
    if (!FIRST) {
#pragma unroll
        for (int k = 0; k < R; k++) job.finish(k, store_J(k), job.mod());
    }
}

// One pass over the tiles of every task.  ROWS: pass B, else pass A.  FIRST:
// the first pass of the transform (reads the job's input, writes its mid
// buffer), else the second (reads mid, writes the job's output).
// LAZY: every task's prime is below LAZY_BOUND (the launcher splits task
// lists by that test); otherwise Harvey butterflies, valid for any prime.
// a radix-8 row pass holds half the registers a thread: one more CTA per SM
template <class Job, int LOGR_ROWS>
constexpr int min_blocks() { return LOGR_ROWS < LOGR ? Job::MIN_BLOCKS + 1 : Job::MIN_BLOCKS; }

template <int LOGN, bool INV, bool ROWS, bool FIRST, bool LAZY, class Job, int LOGR_ROWS = LOGR>
__global__ void __launch_bounds__(256, (min_blocks<Job, LOGR_ROWS>()))
    pass_kernel(const __grid_constant__ typename Job::Params prm)
{
    using C = Cfg<LOGN, LOGR_ROWS>;
    constexpr int TILES = ROWS ? C::ROW_TILES : C::COL_TILES;
    const u32 task = blockIdx.x / TILES;
    const u32 tile = blockIdx.x % TILES;
    Job job(prm, task);
    if (!job.active()) return;
    pass_body<LOGN, INV, ROWS, FIRST, LAZY, Job, LOGR_ROWS>(job, tile);
}

template <int LOGN, bool INV, bool FIRST, int LOGR_ROWS = LOGR>
struct PassShape {
    using C = Cfg<LOGN, LOGR_ROWS>;
    static constexpr bool ROWS = (INV == FIRST); // inverse starts with rows, forward with columns
    static constexpr int threads = ROWS ? C::ROW_THREADS : C::COL_THREADS;
    static constexpr int smem = ROWS ? C::ROW_SMEM : C::COL_SMEM;
    static constexpr int tiles = ROWS ? C::ROW_TILES : C::COL_TILES;
    static constexpr int tile_elems = ROWS ? C::ROW_TILE : C::TILE;
};

// Launch one pass of a transform over `ntasks` tasks.
template <int LOGN, bool INV, bool FIRST, bool LAZY, class Job, int LOGR_ROWS = LOGR>
inline cudaError_t launch_pass_fixed(const typename Job::Params &prm, u32 ntasks, cudaStream_t st, const char *name)
{
    using S = PassShape<LOGN, INV, FIRST, LOGR_ROWS>;
    int extra = Job::EXTRA_WORDS_PER_ELEM;
    if constexpr (Job::RUNTIME_EXTRA) extra = (int)Job::extra_words(prm);
    const int smem = S::smem + extra * S::tile_elems * 8;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (ntasks == 0) return cudaSuccess;
    auto kern = pass_kernel<LOGN, INV, S::ROWS, FIRST, LAZY, Job, LOGR_ROWS>;
    if (smem > 48 * 1024) {
        static int attr = 0; // one instantiation per kernel: raise its opt-in limit when needed
        if (smem > attr) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            attr = smem;
        }
    }
    kern<<<dim3(ntasks * S::tiles), dim3(S::threads), smem, st>>>(prm);
    fheon::prof_mark(st, name);
    return cudaGetLastError();
}

template <bool INV, bool FIRST, bool LAZY, class Job, int LOGR_ROWS>
inline cudaError_t launch_pass_l(u32 logN, const typename Job::Params &prm, u32 ntasks, cudaStream_t st,
                                 const char *name)
{
    switch (logN) {
    case 10: return launch_pass_fixed<10, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    case 11: return launch_pass_fixed<11, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    case 12: return launch_pass_fixed<12, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    case 13: return launch_pass_fixed<13, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    case 14: return launch_pass_fixed<14, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    case 15: return launch_pass_fixed<15, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    case 16: return launch_pass_fixed<16, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    case 17: return launch_pass_fixed<17, INV, FIRST, LAZY, Job, LOGR_ROWS>(prm, ntasks, st, name);
    default: return cudaErrorInvalidValue;
    }
}

// One pass; `lazy` selects the conditional-subtraction-free butterflies, valid
// only when every task's prime is below LAZY_BOUND.  LOGR_ROWS: the radix of a
// row pass (3 or 4; a column pass is radix 16 either way).
template <bool INV, bool FIRST, class Job, int LOGR_ROWS = LOGR>
inline cudaError_t launch_pass(u32 logN, const typename Job::Params &prm, u32 ntasks, cudaStream_t st,
                               const char *name, bool lazy = false)
{
    return lazy ? launch_pass_l<INV, FIRST, true, Job, LOGR_ROWS>(logN, prm, ntasks, st, name)
                : launch_pass_l<INV, FIRST, false, Job, LOGR_ROWS>(logN, prm, ntasks, st, name);
}

// Both passes of a transform whose two passes use the same job type.
template <bool INV, class Job>
inline cudaError_t launch(u32 logN, const typename Job::Params &prm, u32 ntasks, cudaStream_t st)
{
    cudaError_t e = launch_pass<INV, true, Job>(logN, prm, ntasks, st, INV ? "ntt_inv_rows" : "ntt_fwd_cols");
    if (e != cudaSuccess) return e;
    return launch_pass<INV, false, Job>(logN, prm, ntasks, st, INV ? "ntt_inv_cols" : "ntt_fwd_rows");
}

} // namespace ntt
