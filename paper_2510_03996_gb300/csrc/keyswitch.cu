// keyswitch.cu -- the homomorphic rotation: Galois automorphism + hybrid key
// switching (paper Sec. 3.2 rotation, Sec. 6 "4 digits"; Han-Ki hybrid key
// switching with Cheon et al. fast base conversion), for one ciphertext or a
// batch of ciphertexts at mixed levels and Galois elements.
//
// Pipeline of one ciphertext (c0, c1) at level l, Galois element g, beta =
// ceil(l/alpha) digits, everything in the evaluation domain.  Six launches
// cover a whole batch; each is one NTT pass over a task list:
//   IC   INTT of sigma_g(c1): gather on load, last pass scaled by
//        N^-1 * Dhat_i^-1 (the ModUp input scaling)            -> xt[l]
//   UPA  first NTT pass of every new limb of every digit; the load computes
//        the ModUp base conversion from the digit's xt limbs    -> ext[j][t]
//   UPB  second NTT pass, repeated over the digits j of one limb t; each
//        result is multiplied by key_g[j][b][t] and summed in registers
//        (digit limbs of t come straight from sigma_g(c1))      -> acc[2][l+K]
//   DNI  INTT of the P limbs of acc, scaled N^-1 * Phat_k^-1     -> pc[2][K]
//   DNA  first NTT pass of each q_i limb; the load computes the ModDown base
//        conversion P -> q_i from pc                            -> conv[2][l]
//   DNB  second pass; the store forms (acc - conv) * P^-1 and adds
//        sigma_g(c0) to component 0                              -> out[2][l]
// Workspace of one ciphertext (limbs of N u64):
//   xt[l] | ext[beta][l+K] | acc[2][l+K] | pc[2][K] | conv[2][l].
// The key is in Montgomery form, so a product with it reduces to the plain
// residue with one REDC.
//
// Hoisted rotations (the "fast rotations" of paper Sec. 3.2; Halevi-Shoup
// hoisting): rotations of one input share IC, UPA and UPB, run once on c1
// without the automorphism; each rotation's inner product then reads the
// shared raised digits through the sigma_g gather (sigma_g maps every aligned
// block of 2^s evaluation slots onto one aligned block, so the gather stays
// coalesced), and keeps its own acc | pc | conv.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <type_traits>
#include <vector>

#include "jobs.cuh"
#include "tma.cuh"

namespace fheon {

namespace {

struct RotDesc {
    const u64 *c0, *c1; // input components, level limbs each
    u64 *out;           // [2][level][N]
    const u64 *key;     // [beta_max][2][L+K][N], Montgomery form
    u64 *xt;            // INTT of c1, scaled for ModUp [level]
    u64 *ext;           // raised digits [beta][level+K] (shared within a hoisted group)
    u64 *acc;           // acc[2][level+K] | pc[2][K] | conv[2][level]
    u64 g;              // the rotation's Galois element
    u64 gi;             // element applied to c1 on its way into xt (g; 1 when hoisted)
    u64 gx;             // element applied to ext in the inner product (0: none; g when hoisted)
    u32 level, beta;
    const u64 *c1add;   // added to output component 1 (relinearisation: d1), or null
};

struct BatchParams {
    TabPtrs tp;
    const RotDesc *desc; // batch: descriptor per ciphertext (null: `one`)
    const u32 *tasks;    // batch: (ct << 16) | sub per task (null: closed form over `one`)
    RotDesc one;
    u32 L, K, alpha;
    const ulonglong2 *modup_scale;
    const u64 *modup_conv;
    const ulonglong2 *moddown_scale;
    const u64 *moddown_conv;
    const ulonglong2 *pinv;
    int *err; // device error word: FHEON_ERR_TIMEOUT after a wait gave up
};

// ST_UPA_T / ST_DNA_T: tiled base conversions, task sub = (digit or component) << 8 | class
enum Stage { ST_IC, ST_UPA, ST_UPB, ST_DNI, ST_DNA, ST_DNB, ST_UPA_T, ST_DNA_T, ST_COUNT };
// class of a tiled task: 0 / 1 = targets whose prime takes Harvey / lazy
// butterflies; CLS_ALL = every target (closed-form tasks, run with Harvey)
constexpr u32 CLS_ALL = 2;

// (descriptor, sub-index) of a task; closed forms for a single ciphertext
template <int STAGE>
__device__ __forceinline__ const RotDesc &task_of(const BatchParams &P, u32 task, u32 &sub)
{
    if (P.tasks) {
        const u32 w = P.tasks[task];
        sub = w & 0xFFFFu;
        return P.desc[w >> 16];
    }
    const RotDesc &d = P.one;
    const u32 l = d.level, nl = l + P.K, A = P.alpha;
    if (STAGE == ST_UPA) {
        // digits j < beta-1 contribute nl - alpha limbs each, the last nl - d_last
        const u32 full = (d.beta - 1) * (nl - A);
        const u32 j = task < full ? task / (nl - A) : d.beta - 1;
        const u32 r = task - j * (nl - A);
        const u32 dj = min(A, l - j * A);
        sub = (j << 8) | (r < j * A ? r : r + dj);
    } else if (STAGE == ST_UPA_T || STAGE == ST_DNA_T) {
        sub = (task << 8) | CLS_ALL; // every target of the digit | component (Harvey butterflies)
    } else {
        sub = task;
    }
    return d;
}

__device__ __forceinline__ u64 *ws_ext(const RotDesc &d, u32) { return d.ext; }
__device__ __forceinline__ u64 *ws_acc(const RotDesc &d, u32, u32) { return d.acc; }
__device__ __forceinline__ u64 *ws_pc(const RotDesc &d, u32 K, u32 N) { return ws_acc(d, K, N) + (u64)2 * (d.level + K) * N; }
__device__ __forceinline__ u64 *ws_conv(const RotDesc &d, u32 K, u32 N) { return ws_pc(d, K, N) + (u64)2 * K * N; }

struct JobCommon : ntt::JobBase {
    using Params = BatchParams;
    const BatchParams &p;
    const RotDesc *d;
    u32 midx;
    __device__ JobCommon(const BatchParams &P) : p(P) {}
    __device__ bool active() const { return true; }
    __device__ ModConst mod() const { return p.tp.mc[midx]; }
    __device__ const ulonglong2 *twiddles(bool inv) const { return (inv ? p.tp.twi : p.tp.twf) + (u64)midx * p.tp.N; }
    __device__ ulonglong2 inv_scale() const { return make_ulonglong2(0, 0); }
};

// IC: INTT of sigma_g(c1) limb t, scaled for ModUp, into xt[t].  The first
// (row) pass reads the tile's sources, one aligned tile of c1, in order and
// places each at its destination in shared memory (GATHER_LOAD)
struct IcJob : JobCommon {
    const u64 *in;
    u64 *out;
    u64 ginv;
    u32 t;
    __device__ IcJob(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<ST_IC>(P, task, sub);
        t = sub;
        midx = t;
        in = d->c1 + (u64)t * P.tp.N;
        out = d->xt + (u64)t * P.tp.N;
        ginv = inv_odd(d->gi);
    }
    template <bool INV> __device__ u64 load_first(u32 J) const { return in[automorph_src(J, d->gi, p.tp.logN)]; }
    static constexpr bool GATHER_LOAD = true;
    __device__ u32 gather_src(u32 J) const { return automorph_src(J, d->gi, p.tp.logN); }
    __device__ u32 gather_dst(u32 s) const { return automorph_src(s, ginv, p.tp.logN); }
    __device__ u64 load_src(u32 s) const { return in[s]; }
    __device__ u64 load_mid(u32 J) const { return out[J]; }
    __device__ void store_mid(u32 J, u64 v) const { out[J] = v; }
    __device__ ulonglong2 inv_scale() const { return modup_scale(p.modup_scale, t, d->level, p.alpha); }
    __device__ void store_last(int, u32 J, u64 v, const ModConst &) const { out[J] = v; }
};

// UPA: first forward pass of limb t of digit j; the load is the ModUp base
// conversion  y = sum_i xt[d0+i] * (Dhat_i mod m_t) (Montgomery constants, one REDC)
struct UpAJob : JobCommon {
    static constexpr int MIN_BLOCKS = 3;
    const u64 *src;
    const u64 *cf;
    u64 *mid;
    u32 dsz;
    __device__ UpAJob(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<ST_UPA>(P, task, sub);
        const u32 j = sub >> 8, t = sub & 0xFF, l = d->level, A = P.alpha, N = P.tp.N;
        midx = limb_modidx(t, l, P.L);
        const u32 d0 = j * A;
        dsz = min(A, l - d0);
        src = d->xt + (u64)d0 * N;
        cf = P.modup_conv + ((u64)(j * A + (dsz - 1)) * A) * (P.L + P.K) + midx;
        mid = ws_ext(*d, N) + ((u64)j * (l + P.K) + t) * N;
    }
    template <bool INV> __device__ u64 load_first(u32) const { return 0; }
    // sources outermost: one constant per source, 16 independent 128-bit sums
    static constexpr bool TILE_LOAD = true;
    // two halves of 8 elements keep 8 (not 16) 128-bit sums live
    __device__ void load_tile_first(const u32 (&J)[ntt::R], const int (&)[ntt::R], u64 (&x)[ntt::R]) const
    {
        const u32 N = p.tp.N, nm = p.L + p.K;
        const ModConst &m = p.tp.mc[midx];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            u128acc a[ntt::R / 2];
#pragma unroll
            for (int v = 0; v < ntt::R / 2; v++) acc_zero(a[v]);
            for (u32 i = 0; i < dsz; i++) {
                const u64 c = __ldg(&cf[(u64)i * nm]);
                const u64 *s = src + (u64)i * N;
#pragma unroll
                for (int v = 0; v < ntt::R / 2; v++) acc_mad(a[v], s[J[h * 8 + v]], c);
            }
#pragma unroll
            for (int v = 0; v < ntt::R / 2; v++) x[h * 8 + v] = redc_lazy(a[v].hi, a[v].lo, m.q, m.qneg_inv); // [0, 2q): the NTT takes it lazily
        }
    }
    __device__ u64 load_mid(u32 J) const { return mid[J]; }
    __device__ void store_mid(u32 J, u64 v) const { mid[J] = v; }
    __device__ void store_last(int, u32, u64, const ModConst &) const {}
};

// UPB: second forward pass of limb t for every digit j, summed against the key.
// The two running sums of each of the thread's 16 output slots live in shared
// memory (slot k of thread x at k*blockDim + x; only that thread touches it).
struct UpBJob : JobCommon {
    static constexpr int MIN_BLOCKS = 2;
    static constexpr int EXTRA_WORDS_PER_ELEM = 2;
    const u64 *mid, *kb, *ka, *c1t;
    u64 *acc0, *acc1;
    u64 *sacc;
    u32 t, nrep;
    bool pass;
    __device__ void attach(u64 *s) { sacc = s; }
    __device__ u64 &slot(int comp, int k) const
    {
        return sacc[(u64)comp * ntt::R * blockDim.x + (u64)k * blockDim.x + threadIdx.x];
    }
    __device__ UpBJob(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<ST_UPB>(P, task, sub);
        t = sub;
        const u32 l = d->level, N = P.tp.N;
        midx = limb_modidx(t, l, P.L);
        nrep = d->beta;
        c1t = d->c1 + (u64)t * N;
        acc0 = ws_acc(*d, P.K, N) + (u64)t * N;
        acc1 = acc0 + (u64)(l + P.K) * N;
    }
    __device__ int reps() const { return (int)nrep; }
    // this row tile's operands of digit j into L2: the two key tiles, and the
    // mid tile (or, for the digit holding t, the gathered block of sigma_g(c1))
    __device__ void prefetch_rep(u32 j, u32 tile) const
    {
        const u32 l = d->level, N = p.tp.N, nm = p.L + p.K, te = N < 4096 ? N : 4096;
        const u64 off = (u64)tile * te;
        prefetch_l2(d->key + (((u64)j * 2 + 0) * nm + midx) * N + off, te * 8);
        prefetch_l2(d->key + (((u64)j * 2 + 1) * nm + midx) * N + off, te * 8);
        if ((t < l) && (t / p.alpha == j))
            prefetch_l2(c1t + (automorph_src((u32)off, d->g, p.tp.logN) & ~(te - 1)), te * 8);
        else
            prefetch_l2(ws_ext(*d, N) + ((u64)j * (l + p.K) + t) * N + off, te * 8);
    }
    __device__ void begin(int j, u32 tile, u32)
    {
        const u32 l = d->level, N = p.tp.N, nm = p.L + p.K;
        if (j == 0) {
#pragma unroll
            for (int k = 0; k < ntt::R; k++) slot(0, k) = slot(1, k) = 0;
            if (threadIdx.x == 0) prefetch_rep(0, tile);
        }
        if (threadIdx.x == 0 && (u32)j + 1 < nrep) prefetch_rep(j + 1, tile);
        pass = (t < l) && (t / p.alpha == (u32)j);
        mid = ws_ext(*d, N) + ((u64)j * (l + p.K) + t) * N;
        kb = d->key + (((u64)j * 2 + 0) * nm + midx) * N;
        ka = d->key + (((u64)j * 2 + 1) * nm + midx) * N;
    }
    __device__ bool passthrough() const { return pass; }
    __device__ u64 load_passthrough(u32 J) const { return c1t[automorph_src(J, d->g, p.tp.logN)]; }
    template <bool INV> __device__ u64 load_first(u32) const { return 0; }
    __device__ u64 load_mid(u32 J) const { return mid[J]; }
    __device__ void store_mid(u32, u64) const {}
    __device__ void store_last(int k, u32 J, u64 v, const ModConst &m)
    {
        u64 &s0 = slot(0, k), &s1 = slot(1, k);
        s0 = addmod(s0, mulmod_mont(v, __ldg(&kb[J]), m), m.q);
        s1 = addmod(s1, mulmod_mont(v, __ldg(&ka[J]), m), m.q);
    }
    __device__ void finish(int k, u32 J, const ModConst &)
    {
        acc0[J] = slot(0, k);
        acc1[J] = slot(1, k);
    }
};

// DNI: INTT of P limb k of component b of acc, scaled N^-1 * Phat_k^-1, into pc
struct DnIJob : JobCommon {
    const u64 *in;
    u64 *out;
    u32 k;
    __device__ DnIJob(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<ST_DNI>(P, task, sub);
        const u32 b = sub / P.K, l = d->level, N = P.tp.N;
        k = sub % P.K;
        midx = P.L + k;
        in = ws_acc(*d, P.K, N) + ((u64)b * (l + P.K) + l + k) * N;
        out = ws_pc(*d, P.K, N) + ((u64)b * P.K + k) * N;
    }
    template <bool INV> __device__ u64 load_first(u32 J) const { return in[J]; }
    __device__ u64 load_mid(u32 J) const { return out[J]; }
    __device__ void store_mid(u32 J, u64 v) const { out[J] = v; }
    __device__ ulonglong2 inv_scale() const { return p.moddown_scale[k]; }
    __device__ void store_last(int, u32 J, u64 v, const ModConst &) const { out[J] = v; }
};

// DNA: first forward pass of q_i limb of component b; the load is the ModDown
// base conversion P -> q_i from pc
struct DnAJob : JobCommon {
    static constexpr int MIN_BLOCKS = 3;
    const u64 *pc;
    u64 *mid;
    u32 i;
    __device__ DnAJob(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<ST_DNA>(P, task, sub);
        const u32 l = d->level, N = P.tp.N, b = sub / l;
        i = sub % l;
        midx = i;
        pc = ws_pc(*d, P.K, N) + (u64)b * P.K * N;
        mid = ws_conv(*d, P.K, N) + ((u64)b * l + i) * N;
    }
    template <bool INV> __device__ u64 load_first(u32) const { return 0; }
    static constexpr bool TILE_LOAD = true;
    __device__ void load_tile_first(const u32 (&J)[ntt::R], const int (&)[ntt::R], u64 (&x)[ntt::R]) const
    {
        const u32 N = p.tp.N;
        const ModConst &m = p.tp.mc[i];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            u128acc a[ntt::R / 2];
#pragma unroll
            for (int v = 0; v < ntt::R / 2; v++) acc_zero(a[v]);
            for (u32 k = 0; k < p.K; k++) {
                const u64 c = __ldg(&p.moddown_conv[(u64)k * p.L + i]);
                const u64 *s = pc + (u64)k * N;
#pragma unroll
                for (int v = 0; v < ntt::R / 2; v++) acc_mad(a[v], s[J[h * 8 + v]], c);
            }
#pragma unroll
            for (int v = 0; v < ntt::R / 2; v++) x[h * 8 + v] = redc_lazy(a[v].hi, a[v].lo, m.q, m.qneg_inv); // [0, 2q): the NTT takes it lazily
        }
    }
    __device__ u64 load_mid(u32 J) const { return mid[J]; }
    __device__ void store_mid(u32 J, u64 v) const { mid[J] = v; }
    __device__ void store_last(int, u32, u64, const ModConst &) const {}
};

// DNB: second forward pass; out = (acc - conv) * P^-1 (+ sigma_g(c0) for b = 0,
// + c1add for b = 1 when given)
struct DnBJob : JobCommon {
    static constexpr int MIN_BLOCKS = 2;
    const u64 *mid, *acc, *c0i, *c1a;
    u64 *out;
    ulonglong2 pi;
    u32 b;
    __device__ DnBJob(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<ST_DNB>(P, task, sub);
        const u32 l = d->level, N = P.tp.N, i = sub % l;
        b = sub / l;
        midx = i;
        mid = ws_conv(*d, P.K, N) + ((u64)b * l + i) * N;
        acc = ws_acc(*d, P.K, N) + ((u64)b * (l + P.K) + i) * N;
        c0i = d->c0 + (u64)i * N;
        c1a = (b == 1 && d->c1add) ? d->c1add + (u64)i * N : nullptr;
        out = d->out + ((u64)b * l + i) * N;
        pi = P.pinv[i];
    }
    // the row tile's acc and gathered sigma_g(c0) block into L2 while the NTT runs
    __device__ void begin(int, u32 tile, u32 te) const
    {
        if (threadIdx.x != 0) return;
        const u64 off = (u64)tile * te;
        prefetch_l2(acc + off, te * 8);
        if (b == 0) prefetch_l2(c0i + (automorph_src((u32)off, d->g, p.tp.logN) & ~(te - 1)), te * 8);
    }
    template <bool INV> __device__ u64 load_first(u32) const { return 0; }
    __device__ u64 load_mid(u32 J) const { return mid[J]; }
    __device__ void store_mid(u32, u64) const {}
    __device__ void store_last(int, u32 J, u64 y, const ModConst &m) const
    {
        u64 r = shoup(acc[J] + m.q - y, pi.x, pi.y, m.q);
        if (b == 0) r = addmod(r, c0i[automorph_src(J, d->g, p.tp.logN)], m.q);
        else if (c1a) r = addmod(r, c1a[J], m.q);
        out[J] = r;
    }
    // the operands of 8 elements are loaded before any of their stores, so
    // their latencies overlap (a store may alias a later load otherwise)
    static constexpr bool TILE_STORE = true;
    template <int RR>
    __device__ void store_tile_last(const u32 (&J)[RR], const u64 (&y)[RR], const ModConst &m) const
    {
        const bool add = b == 0 || c1a;
#pragma unroll
        for (int h = 0; h < RR / 8; h++) {
            u64 a[8], c[8];
#pragma unroll
            for (int v = 0; v < 8; v++) {
                const u32 j = J[h * 8 + v];
                a[v] = acc[j];
                c[v] = b == 0 ? c0i[automorph_src(j, d->g, p.tp.logN)] : (c1a ? c1a[j] : 0);
            }
#pragma unroll
            for (int v = 0; v < 8; v++) {
                u64 r = shoup(a[v] + m.q - y[h * 8 + v], pi.x, pi.y, m.q);
                if (add) r = addmod(r, c[v], m.q);
                out[J[h * 8 + v]] = r;
            }
        }
    }
};

// Tiled base conversions: one task per (ciphertext, digit j [UP] or component
// b [DN], prime class) and column tile, repeated over every target limb of that
// class.  The sources (the digit's xt limbs, or the K limbs of pc[b]) are read
// from global memory once per tile: each thread keeps its own round-0 elements
// of every source in shared memory (slot s of source i at i*TILE + s) and only
// ever reads its own slots back, so no barrier is needed.  At most
// MAX_SRC sources.  Class 2 (closed-form single-ciphertext tasks) takes every
// target.
constexpr u32 MAX_SRC = 4;

__device__ __forceinline__ bool class_ok(const BatchParams &P, u32 midx, u32 cls)
{
    return cls == CLS_ALL || (u32)(P.tp.mc[midx].q < ntt::LAZY_BOUND) == cls;
}

template <bool UP>
struct TiledConvJob : JobCommon {
    static constexpr int MIN_BLOCKS = 1;
    static constexpr bool RUNTIME_EXTRA = true;
    const u64 *src;  // first source limb (sources are consecutive limbs)
    const u64 *ctab; // UP: modup_conv row of this digit size; DN: moddown_conv
    u64 *midbase;    // UP: ext of digit j; DN: conv of component b
    u64 *mid;
    u64 *xs;
    u64 cf[MAX_SRC];
    u32 nsrc, d0, cls, nrep, cur, rep_now, tile_elems;
    __host__ __device__ static u32 extra_words(const BatchParams &P) { return UP ? P.alpha : P.K; }
    __device__ TiledConvJob(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<UP ? ST_UPA_T : ST_DNA_T>(P, task, sub);
        const u32 l = d->level, N = P.tp.N, A = P.alpha, hi = sub >> 8;
        cls = sub & 0xFF;
        tile_elems = N < 4096 ? N : 4096;
        if (UP) {
            d0 = hi * A;
            nsrc = min(A, l - d0);
            src = d->xt + (u64)d0 * N;
            ctab = P.modup_conv + ((u64)(hi * A + (nsrc - 1)) * A) * (P.L + P.K);
            midbase = ws_ext(*d, N) + (u64)hi * (l + P.K) * N;
        } else {
            d0 = 0;
            nsrc = P.K;
            src = ws_pc(*d, P.K, N) + (u64)hi * P.K * N;
            ctab = P.moddown_conv;
            midbase = ws_conv(*d, P.K, N) + (u64)hi * l * N;
        }
        nrep = 0;
        for (u32 t = 0; t < ntargets(); t++)
            if (is_target(t)) nrep++;
        cur = 0xFFFFFFFFu;
        midx = 0;
    }
    __device__ u32 ntargets() const { return UP ? d->level + p.K : d->level; }
    __device__ bool is_target(u32 t) const
    {
        const u32 l = d->level;
        if (UP && t >= d0 && t < d0 + nsrc) return false;
        return class_ok(p, UP ? limb_modidx(t, l, p.L) : t, cls);
    }
    __device__ void attach(u64 *s) { xs = s; }
    __device__ int reps() const { return (int)nrep; }
    __device__ void begin(int rep, u32, u32)
    {
        rep_now = (u32)rep;
        u32 t = cur + 1;
        while (!is_target(t)) t++;
        cur = t;
        const u32 l = d->level, N = p.tp.N;
        midx = UP ? limb_modidx(t, l, p.L) : t;
        mid = midbase + (u64)t * N;
#pragma unroll
        for (u32 i = 0; i < MAX_SRC; i++)
            if (i < nsrc) cf[i] = UP ? __ldg(&ctab[(u64)i * (p.L + p.K) + midx]) : __ldg(&ctab[(u64)i * p.L + t]);
    }
    template <bool INV> __device__ u64 load_first(u32) const { return 0; }
    static constexpr bool TILE_LOAD = true;
    __device__ void load_tile_first(const u32 (&J)[ntt::R], const int (&S)[ntt::R], u64 (&x)[ntt::R]) const
    {
        const u32 N = p.tp.N;
        u128acc a[ntt::R];
#pragma unroll
        for (int v = 0; v < ntt::R; v++) acc_zero(a[v]);
#pragma unroll
        for (u32 i = 0; i < MAX_SRC; i++) {
            if (i >= nsrc) break;
            u64 *xi = xs + (u64)i * tile_elems;
            if (rep_now == 0) {
                const u64 *s = src + (u64)i * N;
#pragma unroll
                for (int v = 0; v < ntt::R; v++) {
                    const u64 y = s[J[v]];
                    xi[S[v]] = y;
                    acc_mad(a[v], y, cf[i]);
                }
            } else {
#pragma unroll
                for (int v = 0; v < ntt::R; v++) acc_mad(a[v], xi[S[v]], cf[i]);
            }
        }
        const ModConst &m = p.tp.mc[midx];
#pragma unroll
        for (int v = 0; v < ntt::R; v++) x[v] = redc_lazy(a[v].hi, a[v].lo, m.q, m.qneg_inv); // [0, 2q)
    }
    __device__ u64 load_mid(u32 J) const { return mid[J]; }
    __device__ void store_mid(u32 J, u64 v) const { mid[J] = v; }
    __device__ void store_last(int, u32, u64, const ModConst &) const {}
};

// UPB, schedule 1: the plain second forward pass of new limb t of digit j
// (same tasks as UPA), final values back into ext[j][t].  Over a lazy prime
// they stay unreduced (< 36q): the inner product's 128-bit sum of at most 16
// such values times key words (< q) stays below q 2^64 for q < 2^54, so its one
// REDC still returns canonical residues
struct UpB2Job : JobCommon {
    static constexpr bool LAZY_OUT = true;
    u64 *mid;
    __device__ UpB2Job(const BatchParams &P, u32 task) : JobCommon(P)
    {
        u32 sub;
        d = &task_of<ST_UPA>(P, task, sub);
        const u32 j = sub >> 8, t = sub & 0xFF, l = d->level, N = P.tp.N;
        midx = limb_modidx(t, l, P.L);
        mid = ws_ext(*d, N) + ((u64)j * (l + P.K) + t) * N;
    }
    template <bool INV> __device__ u64 load_first(u32) const { return 0; }
    __device__ u64 load_mid(u32 J) const { return mid[J]; }
    __device__ void store_mid(u32, u64) const {}
    __device__ void store_last(int, u32 J, u64 v, const ModConst &) const { mid[J] = v; }
};

// Key inner product, schedule 1: acc_b[t] = sum_j d_j[t] * key[j][b][t] for
// one limb t per task (UPB's tasks), 4 coefficients per thread, 16-byte
// streams of the digits and keys, lazy 128-bit sums and one REDC each.
constexpr int IP_TPB = 256, IP_VEC = 4;
__global__ void __launch_bounds__(IP_TPB) ks_ip_kernel(const __grid_constant__ BatchParams P, u32 chunks)
{
    const u32 task = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    u32 t;
    const RotDesc &d = task_of<ST_UPB>(P, task, t);
    const u32 l = d.level, N = P.tp.N, nm = P.L + P.K, nl = l + P.K;
    const u32 midx = limb_modidx(t, l, P.L);
    const u32 n = (ch * IP_TPB + threadIdx.x) * IP_VEC;
    if (n >= N) return;
    u128acc a0[IP_VEC], a1[IP_VEC];
#pragma unroll
    for (int v = 0; v < IP_VEC; v++) { acc_zero(a0[v]); acc_zero(a1[v]); }
    const u64 *ext = ws_ext(d, N) + (u64)t * N + n;
#pragma unroll 2
    for (u32 j = 0; j < d.beta; j++) {
        u64 x[IP_VEC];
        if (t < l && t / P.alpha == j) {
            const u64 *src = d.c1 + (u64)t * N;
#pragma unroll
            for (int v = 0; v < IP_VEC; v++) x[v] = src[automorph_src(n + v, d.g, P.tp.logN)];
        } else if (d.gx) {
            // hoisted: sigma_g of the shared raised digit
            const u64 *e = ext - n + (u64)j * nl * N;
#pragma unroll
            for (int v = 0; v < IP_VEC; v++) x[v] = e[automorph_src(n + v, d.gx, P.tp.logN)];
        } else {
            const ulonglong2 *e2 = reinterpret_cast<const ulonglong2 *>(ext + (u64)j * nl * N);
#pragma unroll
            for (int v = 0; v < IP_VEC / 2; v++) {
                const ulonglong2 e = e2[v];
                x[2 * v] = e.x;
                x[2 * v + 1] = e.y;
            }
        }
        const ulonglong2 *kb = reinterpret_cast<const ulonglong2 *>(d.key + (((u64)j * 2 + 0) * nm + midx) * N + n);
        const ulonglong2 *ka = reinterpret_cast<const ulonglong2 *>(d.key + (((u64)j * 2 + 1) * nm + midx) * N + n);
#pragma unroll
        for (int v = 0; v < IP_VEC / 2; v++) {
            const ulonglong2 b = __ldcs(kb + v), a = __ldcs(ka + v);
            acc_mad(a0[2 * v], x[2 * v], b.x);
            acc_mad(a0[2 * v + 1], x[2 * v + 1], b.y);
            acc_mad(a1[2 * v], x[2 * v], a.x);
            acc_mad(a1[2 * v + 1], x[2 * v + 1], a.y);
        }
    }
    const ModConst &m = P.tp.mc[midx];
    u64 *o0 = ws_acc(d, P.K, N) + (u64)t * N + n, *o1 = o0 + (u64)nl * N;
#pragma unroll
    for (int v = 0; v < IP_VEC / 2; v++) {
        reinterpret_cast<ulonglong2 *>(o0)[v] =
            make_ulonglong2(redc_acc(a0[2 * v], m.q, m.qneg_inv), redc_acc(a0[2 * v + 1], m.q, m.qneg_inv));
        reinterpret_cast<ulonglong2 *>(o1)[v] =
            make_ulonglong2(redc_acc(a1[2 * v], m.q, m.qneg_inv), redc_acc(a1[2 * v + 1], m.q, m.qneg_inv));
    }
}

// Key inner product, schedule bit 8: per (task, tile of IPB_TE coefficients),
// the operands of each digit -- the digit limb (or the sigma_g block of c1 for
// the digit holding t, or of the shared raised digit when hoisted), and the
// two key limbs -- arrive in shared memory by TMA bulk copies, two digits in
// flight; each thread then sums 8 coefficients with lazy 128-bit products and
// one REDC.  sigma_g maps an aligned block of slots onto one aligned block, so
// a gathered operand is one contiguous copy indexed in shared memory.
constexpr int IPB_TPB = 256, IPB_TE = 2048, IPB_PER = IPB_TE / IPB_TPB, IPB_STAGES = 2;
constexpr u32 IPB_SMEM = IPB_STAGES * 3 * IPB_TE * 8 + 64;

__global__ void __launch_bounds__(IPB_TPB, 2) ks_ip_bulk_kernel(const __grid_constant__ BatchParams P, u32 tiles)
{
    extern __shared__ __align__(128) u64 sm[];
    u64 *bar = sm + IPB_STAGES * 3 * IPB_TE;
    const u32 task = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    u32 t;
    const RotDesc &d = task_of<ST_UPB>(P, task, t);
    const u32 l = d.level, N = P.tp.N, nm = P.L + P.K, nl = l + P.K, logN = P.tp.logN;
    const u32 te = N < (u32)IPB_TE ? N : (u32)IPB_TE, off = tile * te;
    const u32 midx = limb_modidx(t, l, P.L);
    // digit j's x operand: its limb, gather element (0: none) and source block
    auto x_of = [&](u32 j, u64 &g, u32 &base) -> const u64 * {
        const bool pass = t < l && t / P.alpha == j;
        g = pass ? d.g : d.gx;
        base = g ? (automorph_src(off, g, logN) & ~(te - 1)) : off;
        return pass ? d.c1 + (u64)t * N : ws_ext(d, N) + ((u64)j * nl + t) * N;
    };
    auto issue = [&](u32 j) {
        u64 *st = sm + (j % IPB_STAGES) * 3 * IPB_TE;
        u64 g;
        u32 base;
        const u64 *x = x_of(j, g, base);
        u64 *b = &bar[j % IPB_STAGES];
        tma::mbar_arrive_expect_tx(b, 3 * te * 8);
        tma::bulk_g2s(st, x + base, te * 8, b);
        tma::bulk_g2s(st + IPB_TE, d.key + (((u64)j * 2 + 0) * nm + midx) * N + off, te * 8, b);
        tma::bulk_g2s(st + 2 * IPB_TE, d.key + (((u64)j * 2 + 1) * nm + midx) * N + off, te * 8, b);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < IPB_STAGES; s++) tma::mbar_init(&bar[s], 1);
        tma::fence_mbar_init();
        for (u32 j = 0; j < d.beta && j < (u32)IPB_STAGES; j++) issue(j);
    }
    __syncthreads();
    u128acc a0[IPB_PER], a1[IPB_PER];
#pragma unroll
    for (int k = 0; k < IPB_PER; k++) { acc_zero(a0[k]); acc_zero(a1[k]); }
    u32 done = 0; // digits whose copies have landed
    bool ok = true;
    for (u32 j = 0; j < d.beta; j++) {
        u64 *b = &bar[j % IPB_STAGES];
        // the whole CTA agrees on a timeout, so no thread waits at a barrier alone
        ok = __syncthreads_and(tma::mbar_wait(b, (j / IPB_STAGES) & 1));
        if (!ok) break;
        done = j + 1;
        const u64 *st = sm + (j % IPB_STAGES) * 3 * IPB_TE;
        u64 g;
        u32 base;
        x_of(j, g, base);
#pragma unroll
        for (int k = 0; k < IPB_PER; k++) {
            const u32 nl_ = k * IPB_TPB + threadIdx.x;
            if (nl_ >= te) break;
            const u32 xi = g ? automorph_src(off + nl_, g, logN) - base : nl_;
            const u64 x = st[xi];
            acc_mad(a0[k], x, st[IPB_TE + nl_]);
            acc_mad(a1[k], x, st[2 * IPB_TE + nl_]);
        }
        __syncthreads(); // stage free
        if (threadIdx.x == 0 && j + IPB_STAGES < d.beta) {
            tma::fence_proxy_async();
            issue(j + IPB_STAGES);
        }
    }
    if (!ok) {
        // record the timeout, let the copies already issued land, leave the outputs
        if (threadIdx.x == 0) {
            atomicExch(P.err, FHEON_ERR_TIMEOUT);
            for (u32 j = done; j < d.beta && j < done + IPB_STAGES; j++)
                tma::mbar_wait(&bar[j % IPB_STAGES], (j / IPB_STAGES) & 1);
        }
        return;
    }
    const ModConst &m = P.tp.mc[midx];
    u64 *o0 = ws_acc(d, P.K, N) + (u64)t * N + off, *o1 = o0 + (u64)nl * N;
#pragma unroll
    for (int k = 0; k < IPB_PER; k++) {
        const u32 nl_ = k * IPB_TPB + threadIdx.x;
        if (nl_ >= te) break;
        o0[nl_] = redc_acc(a0[k], m.q, m.qneg_inv);
        o1[nl_] = redc_acc(a1[k], m.q, m.qneg_inv);
    }
}

BatchParams batch_params(const fheon_ctx *ctx)
{
    BatchParams P{};
    P.tp = tab_ptrs(ctx);
    P.L = ctx->L;
    P.K = ctx->K;
    P.alpha = ctx->alpha;
    P.modup_scale = ctx->tab.modup_scale.as<ulonglong2>();
    P.modup_conv = ctx->tab.modup_conv.as<u64>();
    P.moddown_scale = ctx->tab.moddown_scale.as<ulonglong2>();
    P.moddown_conv = ctx->tab.moddown_conv.as<u64>();
    P.pinv = ctx->tab.pinv.as<ulonglong2>();
    P.err = ctx->err.as<int>();
    return P;
}

// Task lists of the six stages, each split by modulus class: [s][0] tasks
// whose prime needs Harvey butterflies, [s][1] primes below ntt::LAZY_BOUND.
// Null lists mean closed-form tasks over BatchParams::one (class 0 only).
struct Lists {
    const u32 *t[ST_COUNT][2] = {};
    u32 n[ST_COUNT][2] = {};
};

// One stage of the pipeline over both prime classes.  Schedule bit 16 runs
// the row passes at radix 8 (the fused inner product of schedule bit 1 = 0
// keeps radix 16)
template <bool INV, bool FIRST, class Job>
int stage(fheon_ctx *ctx, BatchParams P, const Lists &ls, int s, const char *name)
{
    Range range(name);
    constexpr bool R8_OK = (INV == FIRST) && !std::is_same<Job, UpBJob>::value; // a row pass
    const bool r8 = R8_OK && (ctx->ks_schedule & 16);
    for (int cls = 0; cls < 2; cls++) {
        if (!ls.n[s][cls]) continue;
        P.tasks = ls.t[s][cls];
        cudaError_t e;
        if constexpr (R8_OK) {
            e = r8 ? ntt::launch_pass<INV, FIRST, Job, 3>(ctx->logN, P, ls.n[s][cls], ctx->stream, name, cls == 1)
                   : ntt::launch_pass<INV, FIRST, Job, 4>(ctx->logN, P, ls.n[s][cls], ctx->stream, name, cls == 1);
        } else {
            e = ntt::launch_pass<INV, FIRST, Job>(ctx->logN, P, ls.n[s][cls], ctx->stream, name, cls == 1);
        }
        FHEON_CUDA(ctx, e);
    }
    return FHEON_OK;
}

// the pipeline's launches over `P`; hoisted groups need the raised digits
// kept, so they always take the streaming inner product
int run_pipeline(fheon_ctx *ctx, const BatchParams &P, const Lists &ls, bool hoisted = false)
{
    int rc;
    if ((rc = stage<true, true, IcJob>(ctx, P, ls, ST_IC, "ic_intt_rows"))) return rc;
    if ((rc = stage<true, false, IcJob>(ctx, P, ls, ST_IC, "ic_intt_cols"))) return rc;
    if (ctx->ks_schedule & 2) {
        if ((rc = stage<false, true, TiledConvJob<true>>(ctx, P, ls, ST_UPA_T, "up_bconv_ntt_cols"))) return rc;
    } else {
        if ((rc = stage<false, true, UpAJob>(ctx, P, ls, ST_UPA, "up_bconv_ntt_cols"))) return rc;
    }
    if ((ctx->ks_schedule & 1) == 0 && !hoisted) {
        if ((rc = stage<false, false, UpBJob>(ctx, P, ls, ST_UPB, "up_ntt_rows_keyip"))) return rc;
    } else {
        if ((rc = stage<false, false, UpB2Job>(ctx, P, ls, ST_UPA, "up_ntt_rows"))) return rc;
        const bool bulk = (ctx->ks_schedule & 8) != 0;
        const u32 chunks = bulk ? (ctx->N + IPB_TE - 1) / IPB_TE : (ctx->N + IP_TPB * IP_VEC - 1) / (IP_TPB * IP_VEC);
        if (bulk) {
            // the kernel's shared-memory opt-in, once per device
            static std::atomic<u64> opted{0};
            int dev = 0;
            FHEON_CUDA(ctx, cudaGetDevice(&dev));
            if (!(opted.load() >> (dev & 63) & 1)) {
                FHEON_CUDA(ctx, cudaFuncSetAttribute(ks_ip_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)IPB_SMEM));
                opted.fetch_or(1ull << (dev & 63));
            }
        }
        Range range("ks_inner");
        for (int cls = 0; cls < 2; cls++) {
            if (!ls.n[ST_UPB][cls]) continue;
            BatchParams Q = P;
            Q.tasks = ls.t[ST_UPB][cls];
            if (bulk)
                ks_ip_bulk_kernel<<<ls.n[ST_UPB][cls] * chunks, IPB_TPB, IPB_SMEM, ctx->stream>>>(Q, chunks);
            else
                ks_ip_kernel<<<ls.n[ST_UPB][cls] * chunks, IP_TPB, 0, ctx->stream>>>(Q, chunks);
            prof_mark(ctx->stream, "ks_inner");
            FHEON_CUDA(ctx, cudaGetLastError());
        }
    }
    if ((rc = stage<true, true, DnIJob>(ctx, P, ls, ST_DNI, "dn_intt_rows"))) return rc;
    if ((rc = stage<true, false, DnIJob>(ctx, P, ls, ST_DNI, "dn_intt_cols"))) return rc;
    if (ctx->ks_schedule & 4) {
        if ((rc = stage<false, true, TiledConvJob<false>>(ctx, P, ls, ST_DNA_T, "dn_bconv_ntt_cols"))) return rc;
    } else {
        if ((rc = stage<false, true, DnAJob>(ctx, P, ls, ST_DNA, "dn_bconv_ntt_cols"))) return rc;
    }
    return stage<false, false, DnBJob>(ctx, P, ls, ST_DNB, "dn_ntt_rows_combine");
}

Lists closed_form_lists(const fheon_ctx *ctx, u32 l)
{
    const u32 K = ctx->K, beta = ctx->beta_at(l);
    Lists ls;
    ls.n[ST_IC][0] = l;
    ls.n[ST_UPA][0] = beta * (l + K) - l;
    ls.n[ST_UPB][0] = l + K;
    ls.n[ST_DNI][0] = 2 * K;
    ls.n[ST_DNA][0] = 2 * l;
    ls.n[ST_DNB][0] = 2 * l;
    ls.n[ST_UPA_T][0] = beta;
    ls.n[ST_DNA_T][0] = 2;
    return ls;
}

} // namespace

// One ciphertext, closed-form tasks: no device plan, no allocation.
int keyswitch_rotate(fheon_ctx *ctx, const u64 *c0, const u64 *c1, u32 l, u64 g, const u64 *key, u64 *ws, u64 *out,
                     const u64 *c1add)
{
    BatchParams P = batch_params(ctx);
    P.desc = nullptr;
    const u32 beta = ctx->beta_at(l);
    u64 *ext = ws + (size_t)l * ctx->N;
    P.one = RotDesc{c0, c1, out, key, ws, ext, ext + (size_t)beta * (l + ctx->K) * ctx->N, g, g, 0, l, beta, c1add};
    return run_pipeline(ctx, P, closed_form_lists(ctx, l));
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
    out->scale = in->scale;
    return keyswitch_rotate(ctx, c0, c1, l, g, it->second.mem.as<u64>(), ws, out->c0());
}

// ---------------------------------------------------------------- batches
// A plan holds the descriptors and the six task lists of one batch in device
// memory; plans are cached by the batch's signature (buffers, levels, keys and
// workspace), so a batch rotated repeatedly uploads its plan once.  The memory
// is shared with callers that keep launches referencing it (captured graphs),
// so evicting a plan from the cache never frees memory a graph still reads.
struct RotPlan {
    std::vector<u64> sig;
    std::shared_ptr<DevMem> mem;
    Lists lists;
    const RotDesc *desc;
    u64 last_use = 0;
};

static std::mutex g_plan_mu;
static std::map<fheon_ctx *, std::vector<RotPlan>> &plan_caches()
{
    static auto *c = new std::map<fheon_ctx *, std::vector<RotPlan>>(); // outlives static teardown
    return *c;
}
// one cache per context, kept in a side table; callers hold g_plan_mu
static std::vector<RotPlan> &plan_cache(fheon_ctx *ctx) { return plan_caches()[ctx]; }

void drop_plans(fheon_ctx *ctx)
{
    std::lock_guard<std::mutex> lk(g_plan_mu);
    plan_caches().erase(ctx);
}

// batch plans kept per context (least recently used goes first)
constexpr size_t PLAN_CACHE = 128;
// a plan is written to the device in chunks carried by the launch parameters
struct PlanChunk {
    static constexpr u32 BYTES = 4000;
    unsigned char b[BYTES];
};
__global__ void plan_write_kernel(const __grid_constant__ PlanChunk c, unsigned char *dst, u32 n)
{
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) dst[i] = c.b[i];
}

// workspace limbs of a key-switching batch: each item's own, less the raised
// digits of the items that read their leader's
static size_t ks_ws_total(const fheon_ctx *ctx, const KsItem *items, u32 n, std::vector<size_t> *off)
{
    size_t total = 0;
    for (u32 i = 0; i < n; i++) {
        const u32 l = items[i].level;
        if (off) (*off)[i] = total;
        total += ctx->ks_ws_limbs(l) - (items[i].lead == i ? 0 : l + (size_t)ctx->beta_at(l) * (l + ctx->K));
    }
    return total;
}

int ks_many(fheon_ctx *ctx, const KsItem *items, uint32_t n, bool hoist, PlanKeep *keep)
{
    if (n == 0) return FHEON_OK;
    Range range(hoist ? "key_switch_batch_hoisted" : "key_switch_batch");
    if (n > 65535) return fail(ctx, FHEON_ERR_ARG, "key-switching batch of %u items", n);
    const u32 N = ctx->N;
    std::vector<size_t> ws_off(n);
    const size_t ws_total = ks_ws_total(ctx, items, n, &ws_off);
    int rc = ensure_workspace(ctx, std::max(ws_total, ctx->ks_ws_limbs(ctx->L) + 2 * (size_t)ctx->L));
    if (rc) return rc;
    u64 *ws = ctx->ws.as<u64>();
    std::vector<u64> sig;
    sig.reserve(7 * (size_t)n + 3);
    sig.push_back((u64)ws);
    sig.push_back(n);
    sig.push_back(hoist);
    for (u32 i = 0; i < n; i++) {
        sig.push_back((u64)items[i].c0 ^ ((u64)items[i].level << 56));
        sig.push_back((u64)items[i].c1);
        sig.push_back((u64)items[i].c1add);
        sig.push_back((u64)items[i].out);
        sig.push_back((u64)items[i].key);
        sig.push_back(items[i].g);
        sig.push_back(items[i].lead);
    }
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto &cache = plan_cache(ctx);
    static u64 tick = 0;
    RotPlan *plan = nullptr;
    for (auto &p : cache)
        if (p.sig == sig) { plan = &p; break; }
    if (!plan) {
        std::vector<RotDesc> desc(n);
        std::vector<u32> t[ST_COUNT][2];
        const u32 L = ctx->L, K = ctx->K, A = ctx->alpha;
        // class of a modulus index: 1 when the lazy butterflies apply
        auto cls = [&](u32 midx) { return ctx->mod[midx] < ntt::LAZY_BOUND ? 1 : 0; };
        auto qp = [&](u32 x, u32 l) { return x < l ? x : L + (x - l); };
        for (u32 i = 0; i < n; i++) {
            const KsItem &it = items[i];
            const u32 l = it.level, beta = ctx->beta_at(l);
            const u64 g = it.g;
            u64 *w = ws + ws_off[i] * N;
            if (it.lead == i) {
                u64 *ext = w + (size_t)l * N;
                desc[i] = RotDesc{it.c0, it.c1, it.out, it.key, w, ext, ext + (size_t)beta * (l + K) * N, g,
                                  hoist ? 1 : g, hoist ? g : 0, l, beta, it.c1add};
            } else {
                const RotDesc &ld = desc[it.lead];
                desc[i] = RotDesc{it.c0, it.c1, it.out, it.key, ld.xt, ld.ext, w, g, 1, g, l, beta, it.c1add};
            }
            const u32 c = i << 16;
            const bool raise = it.lead == i;
            for (u32 x = 0; x < l && raise; x++) t[ST_IC][cls(x)].push_back(c | x);
            for (u32 j = 0; j < beta && raise; j++)
                for (u32 x = 0; x < l + K; x++)
                    if (!(x >= j * A && x < std::min(j * A + A, l))) t[ST_UPA][cls(qp(x, l))].push_back(c | (j << 8) | x);
            for (u32 x = 0; x < l + K; x++) t[ST_UPB][cls(qp(x, l))].push_back(c | x);
            for (u32 x = 0; x < 2 * K; x++) t[ST_DNI][cls(L + x % K)].push_back(c | x);
            for (u32 x = 0; x < 2 * l; x++) t[ST_DNA][cls(x % l)].push_back(c | x);
            for (u32 x = 0; x < 2 * l; x++) t[ST_DNB][cls(x % l)].push_back(c | x);
            // tiled conversions: one task per (digit | component, class) that has a target
            for (u32 j = 0; j < beta && raise; j++)
                for (u32 k = 0; k < 2; k++) {
                    bool any = false;
                    for (u32 x = 0; x < l + K; x++)
                        any = any || (!(x >= j * A && x < std::min(j * A + A, l)) && cls(qp(x, l)) == (int)k);
                    if (any) t[ST_UPA_T][k].push_back(c | (j << 8) | k);
                }
            for (u32 b = 0; b < 2; b++)
                for (u32 k = 0; k < 2; k++) {
                    bool any = false;
                    for (u32 x = 0; x < l; x++) any = any || cls(x) == (int)k;
                    if (any) t[ST_DNA_T][k].push_back(c | (b << 8) | k);
                }
        }
        size_t bytes = n * sizeof(RotDesc);
        size_t off[ST_COUNT][2];
        for (int s = 0; s < ST_COUNT; s++)
            for (int k = 0; k < 2; k++) {
                off[s][k] = bytes;
                bytes += t[s][k].size() * sizeof(u32);
            }
        if (cache.size() >= PLAN_CACHE) {
            auto lru = std::min_element(cache.begin(), cache.end(),
                                        [](const RotPlan &a, const RotPlan &b) { return a.last_use < b.last_use; });
            // its memory goes back stream-ordered (the caching allocator reuses it
            // only for later work on the same stream; cudaFree waits by itself),
            // so queued launches still read it; another stream must wait first
            if (lru->mem && lru->mem->st != ctx->stream) cudaStreamSynchronize(lru->mem->st);
            cache.erase(lru);
        }
        cache.emplace_back();
        plan = &cache.back();
        plan->sig = sig;
        plan->mem = std::make_shared<DevMem>();
        if (!plan->mem->alloc(bytes, ctx->stream)) {
            cache.pop_back();
            return fail(ctx, FHEON_ERR_OOM, "rotation plan (%zu bytes)", bytes);
        }
        std::vector<unsigned char> host(bytes);
        memcpy(host.data(), desc.data(), n * sizeof(RotDesc));
        for (int s = 0; s < ST_COUNT; s++)
            for (int k = 0; k < 2; k++)
                memcpy(host.data() + off[s][k], t[s][k].data(), t[s][k].size() * sizeof(u32));
        // written by kernels whose parameters carry the bytes: the launch copies
        // them, so neither a staging buffer nor a wait is needed
        for (size_t o = 0; o < bytes; o += PlanChunk::BYTES) {
            PlanChunk c;
            const u32 nb = (u32)std::min<size_t>(PlanChunk::BYTES, bytes - o);
            memcpy(c.b, host.data() + o, nb);
            plan_write_kernel<<<1, 256, 0, ctx->stream>>>(c, plan->mem->as<unsigned char>() + o, nb);
            prof_mark(ctx->stream, "plan_write");
            FHEON_CUDA(ctx, cudaGetLastError());
        }
        char *base = plan->mem->as<char>();
        plan->desc = reinterpret_cast<const RotDesc *>(base);
        for (int s = 0; s < ST_COUNT; s++)
            for (int k = 0; k < 2; k++) {
                plan->lists.t[s][k] = reinterpret_cast<const u32 *>(base + off[s][k]);
                plan->lists.n[s][k] = (u32)t[s][k].size();
            }
    }
    plan->last_use = ++tick;
    if (keep) keep->push_back(plan->mem);
    BatchParams P = batch_params(ctx);
    P.desc = plan->desc;
    return run_pipeline(ctx, P, plan->lists, hoist);
}


int rotate_many(fheon_ctx *ctx, const fheon_rot_item *items, uint32_t n, bool hoist, PlanKeep *keep)
{
    if (n == 0) return FHEON_OK;
    if (n > 65535) {
        // (an input whose rotations fall in two chunks is raised once per chunk)
        for (u32 s = 0; s < n; s += 65535) {
            int rc = rotate_many(ctx, items + s, std::min<u32>(65535, n - s), hoist, keep);
            if (rc) return rc;
        }
        return FHEON_OK;
    }
    const u32 N = ctx->N;
    // validate and size outputs; lead = the item whose raised digits an item
    // reads (itself, unless it shares a hoisted input)
    std::vector<KsItem> ks(n);
    std::map<const fheon_ct *, u32> first;
    for (u32 i = 0; i < n; i++) {
        const fheon_ct *in = items[i].in;
        fheon_ct *out = items[i].out;
        if (!in || !out) return fail(ctx, FHEON_ERR_ARG, "null ciphertext in batch item %u", i);
        const u64 g = fheon_galois_elt(ctx, items[i].step);
        auto it = ctx->keys.find(g);
        if (it == ctx->keys.end())
            return fail(ctx, FHEON_ERR_NO_KEY, "no rotation key for step %d (batch item %u)", items[i].step, i);
        ks[i].key = it->second.mem.as<u64>();
        ks[i].g = g;
        ks[i].level = in->level;
        ks[i].lead = hoist ? first.emplace(in, i).first->second : i;
    }
    {
        std::set<const fheon_ct *> ins, outs;
        for (u32 i = 0; i < n; i++) ins.insert(items[i].in);
        for (u32 i = 0; i < n; i++) {
            if (ins.count(items[i].out)) return fail(ctx, FHEON_ERR_ARG, "batch output %u aliases an input", i);
            if (!outs.insert(items[i].out).second) return fail(ctx, FHEON_ERR_ARG, "batch output %u repeated", i);
        }
    }
    if (!ctx->batching) {
        // the plain path: one rotation at a time, none hoisted
        for (u32 i = 0; i < n; i++) {
            int rc = rotate_one(ctx, items[i].in, ks[i].g, items[i].out);
            if (rc) return rc;
        }
        return FHEON_OK;
    }
    for (u32 i = 0; i < n; i++) {
        int rc = ct_reshape(ctx, items[i].out, items[i].in->level);
        if (rc) return rc;
        items[i].out->scale = items[i].in->scale;
        ks[i].c0 = items[i].in->c0();
        ks[i].c1 = items[i].in->c1(N);
        ks[i].c1add = nullptr;
        ks[i].out = items[i].out->c0();
    }
    return ks_many(ctx, ks.data(), n, hoist, keep);
}

int mul_relin_many(fheon_ctx *ctx, const RelinItem *items, uint32_t n, PlanKeep *keep)
{
    if (n == 0) return FHEON_OK;
    if (n == 1) return mul_relin_at(ctx, items[0].a, items[0].b, items[0].level, items[0].twice, items[0].out);
    if (!ctx->batching) {
        for (u32 i = 0; i < n; i++) {
            const RelinItem &r = items[i];
            if (!r.a || !r.b || !r.out || r.out == r.a || r.out == r.b)
                return fail(ctx, FHEON_ERR_ARG, "product batch item %u: null or aliased ciphertext", i);
            int rc = mul_relin_at(ctx, r.a, r.b, r.level, r.twice, r.out);
            if (rc) return rc;
        }
        return FHEON_OK;
    }
    auto kit = ctx->keys.find(0);
    if (kit == ctx->keys.end()) return fail(ctx, FHEON_ERR_NO_KEY, "no relinearisation key");
    const u32 N = ctx->N;
    std::vector<KsItem> ks(n);
    size_t tens = 0;
    for (u32 i = 0; i < n; i++) {
        const RelinItem &r = items[i];
        if (!r.a || !r.b || !r.out || r.out == r.a || r.out == r.b)
            return fail(ctx, FHEON_ERR_ARG, "product batch item %u: null or aliased ciphertext", i);
        if (r.level < 1 || r.level > r.a->level || r.level > r.b->level)
            return fail(ctx, FHEON_ERR_LEVEL, "product batch item %u: level %u", i, r.level);
        // an output is resized before later items' operands are read: it may
        // be no item's operand, nor another item's output
        for (u32 j = 0; j < n; j++) {
            if (items[j].a == r.out || items[j].b == r.out)
                return fail(ctx, FHEON_ERR_ARG, "product batch output %u is an operand of item %u", i, j);
            if (j < i && items[j].out == r.out) return fail(ctx, FHEON_ERR_ARG, "product batch output %u repeated", i);
        }
        ks[i].level = r.level;
        ks[i].lead = i;
        tens += 3 * (size_t)r.level;
    }
    // the tensors sit past the batch's key-switching workspace
    const size_t base = std::max(ks_ws_total(ctx, ks.data(), n, nullptr), ctx->ks_ws_limbs(ctx->L) + 2 * (size_t)ctx->L);
    int rc = ensure_workspace(ctx, base + tens);
    if (rc) return rc;
    u64 *d = ctx->ws.as<u64>() + base * N;
    for (u32 i = 0; i < n; i++) {
        const RelinItem &r = items[i];
        const u32 l = r.level;
        const double sc = r.a->scale * r.b->scale;
        FHEON_CUDA(ctx, k_tensor(ctx, r.a->c0(), r.a->c1(N), r.b->c0(), r.b->c1(N), d, l, r.twice));
        if ((rc = ct_reshape(ctx, r.out, l))) return rc;
        r.out->scale = sc;
        // key-switch d2 from s^2 to s (g = 1); d0 joins component 0, d1 component 1
        ks[i].c0 = d;
        ks[i].c1 = d + (size_t)2 * l * N;
        ks[i].c1add = d + (size_t)l * N;
        ks[i].out = r.out->c0();
        ks[i].key = kit->second.mem.as<u64>();
        ks[i].g = 1;
        d += (size_t)3 * l * N;
    }
    return ks_many(ctx, ks.data(), n, false, keep);
}

int rotate_hoisted(fheon_ctx *ctx, const fheon_ct *in, const int32_t *steps, uint32_t n, fheon_ct *const *outs,
                   PlanKeep *keep)
{
    std::vector<fheon_rot_item> items(n);
    for (u32 i = 0; i < n; i++) items[i] = fheon_rot_item{in, outs[i], steps[i]};
    return rotate_many(ctx, items.data(), n, true, keep);
}

} // namespace fheon

namespace {
// one thread arms a TMA barrier for 16 bytes that no copy brings, then waits
// with the library's bounded wait: it gives up after `polls` polls and
// records the timeout in the device error word, as the inner product does
__global__ void wait_selftest_kernel(int *err, u32 polls)
{
    __shared__ __align__(8) u64 bar;
    if (threadIdx.x != 0) return;
    tma::mbar_init(&bar, 1);
    tma::fence_mbar_init();
    tma::mbar_arrive_expect_tx(&bar, 16);
    if (!tma::mbar_wait(&bar, 0, polls)) atomicExch(err, FHEON_ERR_TIMEOUT);
}
} // namespace

extern "C" int fheon_selftest_wait(fheon_ctx *ctx, uint32_t polls)
{
    if (!ctx || polls < 1 || polls > tma::WAIT_POLLS) return FHEON_ERR_ARG;
    wait_selftest_kernel<<<1, 32, 0, ctx->stream>>>(ctx->err.as<int>(), polls);
    FHEON_CUDA(ctx, cudaGetLastError());
    return FHEON_OK;
}

