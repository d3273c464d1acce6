// params.cpp -- host arithmetic for context set-up: NTT-friendly primes, roots
// of unity, Shoup and Montgomery constants, the Gaussian CDT.  None of this
// runs per operation; it fills the constant tables the kernels read.
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace fheon {

typedef unsigned __int128 u128;

u64 h_mulmod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

u64 h_powmod(u64 b, u64 e, u64 m)
{
    u64 acc = 1 % m, base = b % m;
    for (; e; e >>= 1) {
        if (e & 1) acc = h_mulmod(acc, base, m);
        base = h_mulmod(base, base, m);
    }
    return acc;
}

u64 h_invmod(u64 a, u64 m) { return h_powmod(a, m - 2, m); } // m prime

// Miller-Rabin with a fixed witness set that is exact for all 64-bit inputs.
static bool mr_witness(u64 n, u64 a, u64 d, int s)
{
    u64 x = h_powmod(a, d, n);
    if (x == 1 || x == n - 1) return false;
    for (int r = 1; r < s; r++) {
        x = h_mulmod(x, x, n);
        if (x == n - 1) return false;
    }
    return true; // a proves n composite
}
bool h_is_prime(u64 n)
{
    const u64 W[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : W)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; ++s; }
    for (u64 a : W)
        if (mr_witness(n, a, d, s)) return false;
    return true;
}

// Smallest primitive 2N-th root of unity mod q: any root psi0 of X^N = -1,
// then the least of its odd powers.
u64 h_min_root(u64 q, u32 N)
{
    const u64 M = 2ull * N, ex = (q - 1) / M;
    u64 psi0 = 0;
    for (u64 x = 2;; ++x) {
        psi0 = h_powmod(x, ex, q);
        if (h_powmod(psi0, N, q) == q - 1) break;
    }
    const u64 step = h_mulmod(psi0, psi0, q);
    u64 best = psi0, cur = psi0;
    for (u64 k = 1; k < N; ++k) {
        cur = h_mulmod(cur, step, q);
        if (cur < best) best = cur;
    }
    return best;
}

u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

ModConst h_modconst(u64 q)
{
    ModConst c;
    c.q = q;
    u64 inv = q; // Newton iteration for q^-1 mod 2^64 (q odd): 3 -> 6 -> ... -> 96 correct bits
    for (int i = 0; i < 5; i++) inv *= 2 - q * inv;
    c.qneg_inv = 0 - inv;
    c.r1 = (0 - q) % q; // 2^64 mod q
    c.r2 = h_mulmod(c.r1, c.r1, q);
    c.r1_sh = h_shoup(c.r1, q);
    c.twoq = 2 * q;
    c.one_sh = h_shoup(1, q);
    return c;
}

// For each size in order: the largest unused prime below 2^bits that is 1 mod 2N.
bool h_pick_primes(u32 N, const std::vector<u32> &bits, std::vector<u64> &out)
{
    out.clear();
    const u64 M = 2ull * N;
    for (u32 b : bits) {
        if (b < 20 || b > 61) return false;
        const u64 hi = (b == 64) ? ~0ull : ((1ull << b) - 1);
        u64 c = hi - (hi - 1) % M; // largest value <= hi congruent to 1 mod M
        bool ok = false;
        for (; c > (1ull << (b - 1)); c -= M) {
            bool used = false;
            for (u64 u : out) used = used || (u == c);
            if (!used && h_is_prime(c)) { ok = true; break; }
        }
        if (!ok) return false;
        out.push_back(c);
    }
    return true;
}

// Discrete Gaussian CDT, exactly the binary64 evaluation order the scheme
// fixes: rho(k) = exp(-(k*k) / (2 sigma sigma)) for k = -tail..tail, S their
// sum in increasing k, T[k+tail] = (u64) ldexp(partial_sum(k) / S, 64).
void h_cdt_table(double sigma, int tail, u64 *T)
{
    const int n = 2 * tail + 1;
    std::vector<double> rho(n);
    double S = 0.0;
    for (int i = 0; i < n; i++) {
        const int k = i - tail;
        rho[i] = std::exp(-(double)(k * k) / (2.0 * sigma * sigma));
        S += rho[i];
    }
    double part = 0.0;
    for (int i = 0; i < n - 1; i++) {
        part += rho[i];
        T[i] = (u64)std::ldexp(part / S, 64);
    }
    T[n - 1] = 0;
}

} // namespace fheon
