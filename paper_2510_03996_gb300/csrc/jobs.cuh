// jobs.cuh -- NTT job policies over plain limb arrays: where a transform reads
// its limb, which modulus the limb belongs to, and where the result goes.
#pragma once
#include "internal.h"
#include "ntt_core.cuh"

namespace fheon {

// Tables every job needs.
struct TabPtrs {
    const ModConst *mc;
    const ulonglong2 *twf, *twi, *ninv;
    u32 N, logN;
};
inline TabPtrs tab_ptrs(const fheon_ctx *c)
{
    return TabPtrs{c->tab.mc.as<ModConst>(), c->tab.tw_fwd.as<ulonglong2>(), c->tab.tw_inv.as<ulonglong2>(),
                   c->tab.ninv.as<ulonglong2>(), c->N, c->logN};
}

// Scale applied by the last inverse pass.
enum ScaleMode : u32 {
    SCALE_NINV = 0,    // N^-1
    SCALE_MODUP = 1,   // N^-1 * Dhat_i^-1 (ModUp source limb i of its digit at `level`)
    SCALE_MODDOWN = 2, // N^-1 * Phat_k^-1 (P limb k)
};

__device__ __forceinline__ u32 limb_modidx(u32 t, u32 level, u32 L) { return t < level ? t : L + (t - level); }

// N^-1 * Dhat_i^-1 for limb t of its digit at `level`
__device__ __forceinline__ ulonglong2 modup_scale(const ulonglong2 *tab, u32 t, u32 level, u32 A)
{
    const u32 j = t / A, d = min(A, level - j * A);
    return tab[(j * A + (d - 1)) * A + (t - j * A)];
}

// Limbs of a batch of polynomials: limb position p of polynomial `poly` sits at
// base + poly*poly_stride + p*N; its limb index is t = p + first_t, and limb
// index t < level is modulus q_t, otherwise special modulus p_{t-level}
// (modulus index L + t - level).  The first pass writes `out` (the mid
// buffer), the second reads and overwrites it.
struct MapParams {
    TabPtrs tp;
    const u64 *in;
    u64 *out;
    u64 in_poly_stride, out_poly_stride;
    u32 per_poly, first_t, level, L, alpha;
    u64 gather_g;   // inverse first pass only: read in[sigma_g source] (0 = none)
    u32 scale_mode; // ScaleMode
    const ulonglong2 *scale_tab;
};

struct MapJob : ntt::JobBase {
    using Params = MapParams;
    const MapParams &p;
    const u64 *in;
    u64 *out;
    u32 midx, t;
    __device__ MapJob(const MapParams &P, u32 task) : p(P)
    {
        const u32 poly = task / P.per_poly, pos = task % P.per_poly;
        t = pos + P.first_t;
        midx = limb_modidx(t, P.level, P.L);
        in = P.in + poly * P.in_poly_stride + (u64)pos * P.tp.N;
        out = P.out + poly * P.out_poly_stride + (u64)pos * P.tp.N;
    }
    __device__ bool active() const { return true; }
    __device__ ModConst mod() const { return p.tp.mc[midx]; }
    __device__ const ulonglong2 *twiddles(bool inv) const { return (inv ? p.tp.twi : p.tp.twf) + (u64)midx * p.tp.N; }
    template <bool INV> __device__ u64 load_first(u32 J) const
    {
        if (INV && p.gather_g) return in[automorph_src(J, p.gather_g, p.tp.logN)];
        return in[J];
    }
    __device__ u64 load_mid(u32 J) const { return out[J]; }
    __device__ void store_mid(u32 J, u64 v) const { out[J] = v; }
    __device__ ulonglong2 inv_scale() const
    {
        if (p.scale_mode == SCALE_MODUP) return modup_scale(p.scale_tab, t, p.level, p.alpha);
        if (p.scale_mode == SCALE_MODDOWN) return p.scale_tab[t - p.level];
        return p.tp.ninv[midx];
    }
    __device__ void store_last(int, u32 J, u64 v, const ModConst &) const { out[J] = v; }
};

inline MapParams map_params(const fheon_ctx *c, const u64 *in, u64 *out, u32 per_poly, u32 first_t, u32 level)
{
    MapParams m{};
    m.tp = tab_ptrs(c);
    m.in = in;
    m.out = out;
    m.in_poly_stride = (u64)per_poly * c->N;
    m.out_poly_stride = (u64)per_poly * c->N;
    m.per_poly = per_poly;
    m.first_t = first_t;
    m.level = level;
    m.L = c->L;
    m.alpha = c->alpha;
    m.gather_g = 0;
    m.scale_mode = SCALE_NINV;
    m.scale_tab = nullptr;
    return m;
}

} // namespace fheon
