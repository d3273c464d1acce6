// modarith.cuh -- 64-bit modular arithmetic for the sm_103a kernels.
//
// Every step of the rotation path is exact arithmetic modulo word-size primes
// q < 2^61.  There is no 64x64 multiplier on the GPU: a low product is three
// 32-bit IMADs and __umul64hi about six, so the helpers below are chosen to
// spend as few of them as possible:
//   * fixed-operand products (NTT twiddles, scaling constants) use Shoup's
//     precomputed quotient w' = floor(w * 2^64 / q): one high and two low
//     products, result in [0, 2q) for any 64-bit input (Shoup, NTL; the lazy
//     form is the one Harvey's NTT uses);
//   * variable products (key inner product, base conversion, plaintext
//     products) accumulate full 128-bit products and reduce once with
//     Montgomery's REDC (Montgomery 1985): t = (x + m q) / 2^64 with
//     m = x_lo * (-q^-1) mod 2^64, which is x * 2^-64 mod q in [0, 2q) when
//     x < q * 2^64.  One operand carries the 2^64 factor (a constant stored
//     in Montgomery form), so the result is the plain residue;
//   * NTT butterflies are Harvey's lazy ones (Harvey 2014): forward values
//     in [0, 4q), inverse values in [0, 2q), which needs 4q < 2^64.
#pragma once
#include <cstdint>

typedef unsigned long long u64;
typedef unsigned int u32;

// Per-modulus constants read by the kernels.
struct ModConst {
    u64 q;        // the prime
    u64 qneg_inv; // -q^-1 mod 2^64 (REDC)
    u64 r2;       // 2^128 mod q: redc(x * r2) = x * 2^64 mod q (to Montgomery form)
    u64 r1;       // 2^64 mod q
    u64 r1_sh;    // Shoup companion of r1: redc result times r1 = plain residue
    u64 twoq;     // 2q
    u64 one_sh;   // floor(2^64 / q): Shoup product by 1 reduces any word to [0, 2q)
};

__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

// w * y mod q, lazily in [0, 2q), for any y < 2^64 (Shoup).
__device__ __forceinline__ u64 shoup_lazy(u64 y, u64 w, u64 wsh, u64 q)
{
    u64 qh = __umul64hi(wsh, y);
    return w * y - qh * q;
}
__device__ __forceinline__ u64 shoup(u64 y, u64 w, u64 wsh, u64 q)
{
    u64 r = shoup_lazy(y, w, wsh, q);
    return r >= q ? r - q : r;
}

// 128-bit accumulator
struct u128acc {
    u64 lo, hi;
};
__device__ __forceinline__ void acc_zero(u128acc &a) { a.lo = 0; a.hi = 0; }
// a += x * y (128-bit), with the carry chained through the PTX carry flag
__device__ __forceinline__ void acc_mad(u128acc &a, u64 x, u64 y)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(a.lo), "+l"(a.hi)
        : "l"(x), "l"(y));
}
// REDC of (hi:lo) < q * 2^64: (hi:lo) * 2^-64 mod q, in [0, 2q).
// lo + m*q vanishes modulo 2^64, so its carry into the high word is (lo != 0).
__device__ __forceinline__ u64 redc_lazy(u64 hi, u64 lo, u64 q, u64 qneg_inv)
{
    u64 m = lo * qneg_inv;
    return hi + __umul64hi(m, q) + (lo != 0 ? 1ull : 0ull);
}
__device__ __forceinline__ u64 redc(u64 hi, u64 lo, u64 q, u64 qneg_inv)
{
    u64 t = redc_lazy(hi, lo, q, qneg_inv);
    return t >= q ? t - q : t;
}
__device__ __forceinline__ u64 redc_acc(const u128acc &a, u64 q, u64 qneg_inv) { return redc(a.hi, a.lo, q, qneg_inv); }

// x * y mod q for x, y < q (y plain): REDC then a Shoup multiply by 2^64 mod q.
__device__ __forceinline__ u64 mulmod_plain(u64 x, u64 y, const ModConst &m)
{
    u64 t = redc_lazy(__umul64hi(x, y), x * y, m.q, m.qneg_inv);
    return shoup(t, m.r1, m.r1_sh, m.q);
}
// x * ym mod q for x < q and ym = y * 2^64 mod q (Montgomery form).
__device__ __forceinline__ u64 mulmod_mont(u64 x, u64 ym, const ModConst &m)
{
    return redc(__umul64hi(x, ym), x * ym, m.q, m.qneg_inv);
}
__device__ __forceinline__ u64 to_mont(u64 x, const ModConst &m) { return mulmod_mont(x, m.r2, m); }

__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q)
{
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
__device__ __forceinline__ u64 reduce4q(u64 x, u64 q)
{
    u64 tq = q + q;
    x = x >= tq ? x - tq : x;
    return x >= q ? x - q : x;
}
__device__ __forceinline__ u64 reduce2q(u64 x, u64 q) { return x >= q ? x - q : x; }

// Harvey forward (Cooley-Tukey) butterfly: X, Y in [0, 4q) -> [0, 4q).
__device__ __forceinline__ void ct_butterfly(u64 &X, u64 &Y, u64 w, u64 wsh, u64 q, u64 twoq)
{
    u64 x = X >= twoq ? X - twoq : X;
    u64 t = shoup_lazy(Y, w, wsh, q);
    X = x + t;
    Y = x - t + twoq;
}
// Harvey inverse (Gentleman-Sande) butterfly: X, Y in [0, 2q) -> [0, 2q).
__device__ __forceinline__ void gs_butterfly(u64 &X, u64 &Y, u64 w, u64 wsh, u64 q, u64 twoq)
{
    u64 s = X + Y;
    u64 d = X - Y + twoq;
    X = s >= twoq ? s - twoq : s;
    Y = shoup_lazy(d, w, wsh, q);
}

// Bulk prefetch of [p, p + bytes) into L2 (address and size multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, u32 bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// inverse of an odd g modulo 2^64 (Newton's iteration x <- x (2 - g x) doubles
// the number of correct low bits; x = g is right to 3 bits)
__device__ __forceinline__ u64 inv_odd(u64 g)
{
    u64 x = g;
#pragma unroll
    for (int i = 0; i < 5; i++) x *= 2 - g * x;
    return x;
}

// bit reversal of the low `bits` bits
__device__ __forceinline__ u32 brev_bits(u32 x, u32 bits) { return __brev(x) >> (32 - bits); }

// Evaluation-domain Galois automorphism: index j of sigma_g(a) holds index
// src of a, where 2*brv(src)+1 = (2*brv(j)+1) * g mod 2N.  The map by g^-1 is
// its inverse.  It takes an aligned block of 2^b indices (fixed high bits)
// onto an aligned block: the low logN - b bits of brv(j) are fixed, odd
// multiples keep them fixed modulo 2^(logN-b+1), so the high bits of src are
// fixed too.
__device__ __forceinline__ u32 automorph_src(u32 j, u64 g, u32 logN)
{
    u32 k = brev_bits(j, logN);
    u64 twoN = 2ull << logN;
    u64 e = ((2ull * k + 1ull) * g) & (twoN - 1);
    return brev_bits((u32)((e - 1) >> 1), logN);
}
