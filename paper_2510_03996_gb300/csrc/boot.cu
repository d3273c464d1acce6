// boot.cu -- CKKS bootstrapping as a layer.  The paper offers it as a layer
// placed anywhere in a network (the "Bootstrapping Layer" among its support
// functions; its evaluation bootstraps before every ReLU but the first two,
// before the second pooling layer and before the global pooling) and takes
// the algorithm from its library.  This is the published full-slot
// bootstrapping (Cheon, Han, Kim, Kim, Song 2018) with the slot transforms
// factored into the butterfly stages of the special FFT and applied as
// baby-step/giant-step rotation sums (Chen, Chillotti, Song 2019), and the
// modular reduction as a scaled cosine followed by double-angle steps (Han,
// Ki 2020).  Every step runs on the device operations of this library:
//
//   1. ModRaise: limb q_0 of the input to coefficients, centred, into all L
//      primes (mod_raise_ct); it decrypts to t = m + q_0 I, |I| < K.  The
//      raised ciphertext is given scale q_0: its slots are F(t_lo + i t_hi)/q_0.
//   2. CoeffToSlot: the inverse butterfly stages of F (top stages first),
//      merged into `cts_levels` rotation-sum layers, 1/(2K) folded into the
//      first: (t_lo + i t_hi) / (2 K q_0) in bit-reversed slot order.
//   3. With the conjugate c' (Galois element 2N - 1): re = c + c',
//      im = (c' - c) X^(N/2), holding t_lo / (K q_0) and t_hi / (K q_0).
//   4. EvalMod on each: the Chebyshev series of cos(2 pi (K x - 1/4) / 2^r),
//      then r steps c <- 2 c^2 - 1: sin(2 pi t / q_0) ~= 2 pi m / q_0.
//   5. re + im X^(N/2).
//   6. SlotToCoeff: the butterfly stages of F (low stages first), merged into
//      `stc_levels` layers, q_0 / (2 pi Delta_in) folded into the first; the
//      last is encoded so that the output lands on scale ~= Delta_in.
//
// Sparse bootstrap (slots [0, n_s), n_s <= N/4, copies = N / (2 n_s)): the
// input is masked to those slots at level 2 and repeated in every copy of
// n_s slots (its polynomial then lies in Z[X^copies]); after ModRaise the
// trace (the sum of the copies' rotations) keeps copies x the coefficients of
// that subring; CoeffToSlot is the n_s-slot transform in every copy, ending
// in the factor 1 / -i on even / odd copies, so y + conj(y) carries the low
// and the high coefficients in one ciphertext: one EvalMod; SlotToCoeff
// starts with (a, b) -> a + i b in every copy.
//
// Stage of half-length h of F (blocks of 2h slots, u < h the position in the
// block, w_u = exp(2 pi i (5^u mod 8h) / 8h)):
//   out[b+u] = in[b+u] + w_u in[b+u+h],  out[b+u+h] = in[b+u] - w_u in[b+u+h];
// as slot diagonals (out = sum_o d_o Rot_o(in)) it has offsets 0, +h and -h.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <vector>

#include "layer.h"

using namespace fheon;

namespace {

u64 powmod_small(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = (r * b) % m;
        b = (b * b) % m;
        e >>= 1;
    }
    return r;
}

Diags stage(u32 n, u32 h, bool inverse)
{
    const u32 m = 2 * h;
    std::vector<cd> d0(n), dp(n), dm(n);
    for (u32 j = 0; j < n; j++) {
        const u32 u = j % m;
        const bool lo = u < h;
        const u64 e = powmod_small(5, lo ? u : u - h, 4ull * m);
        const double a = 2.0 * M_PI * (double)e / (double)(4ull * m);
        const cd w(std::cos(a), std::sin(a));
        if (!inverse) {
            d0[j] = lo ? cd(1.0) : -w;
            dp[j] = lo ? w : cd(0.0);
            dm[j] = lo ? cd(0.0) : cd(1.0);
        } else {
            d0[j] = lo ? cd(0.5) : -0.5 / w;
            dp[j] = lo ? cd(0.5) : cd(0.0);
            dm[j] = lo ? cd(0.0) : 0.5 / w;
        }
    }
    Diags out;
    auto put = [&](u32 o, const std::vector<cd> &d) {
        auto it = out.find(o);
        if (it == out.end()) {
            out.emplace(o, d);
        } else {
            for (u32 j = 0; j < n; j++) it->second[j] += d[j];
        }
    };
    put(0, d0);
    put(h % n, dp);
    put((n - h % n) % n, dm);
    return out;
}

// A.B (B applied first): (A B v)[j] = sum_a A_a[j] (B v)[j + a]
Diags compose(const Diags &A, const Diags &B, u32 n)
{
    Diags C;
    for (const auto &a : A)
        for (const auto &b : B) {
            const u32 c = (a.first + b.first) % n;
            auto it = C.find(c);
            if (it == C.end()) it = C.emplace(c, std::vector<cd>(n, cd(0.0))).first;
            for (u32 j = 0; j < n; j++) it->second[j] += a.second[j] * b.second[(j + a.first) % n];
        }
    return C;
}

// stages 1..logn split into `levels` consecutive groups, the larger ones at the top
std::vector<std::vector<u32>> stage_groups(u32 logn, u32 levels)
{
    std::vector<std::vector<u32>> g(levels);
    const u32 base = logn / levels, extra = logn % levels;
    u32 s = 1;
    for (u32 i = 0; i < levels; i++) {
        const u32 sz = base + (i >= levels - extra ? 1 : 0);
        for (u32 k = 0; k < sz; k++) g[i].push_back(s++);
    }
    return g;
}

struct MergedLevel {
    u32 stride;
    Diags M;
};

std::vector<MergedLevel> merged_levels(u32 n, u32 levels, bool cts)
{
    u32 logn = 0;
    while ((1u << logn) < n) logn++;
    auto groups = stage_groups(logn, levels);
    if (cts) std::reverse(groups.begin(), groups.end());
    std::vector<MergedLevel> out;
    for (auto &g : groups) {
        if (cts) std::reverse(g.begin(), g.end()); // top stage of the group first
        Diags M;
        bool first = true;
        for (u32 s : g) {
            Diags S = stage(n, 1u << (s - 1), cts);
            M = first ? S : compose(S, M, n);
            first = false;
        }
        out.push_back(MergedLevel{1u << (std::min(g.front(), g.back()) - 1), std::move(M)});
    }
    return out;
}

// An n_s-slot map as an n-slot map for inputs that repeat every n_s slots:
// every diagonal tiled n / n_s times, offset o taken as o or o - n_s (the
// nearer to 0) modulo n.  On such an input it is the n_s-slot map in every copy.
Diags replicate(const Diags &M, u32 ns, u32 n)
{
    Diags out;
    for (const auto &kv : M) {
        const u32 o = kv.first <= ns / 2 ? kv.first : (u32)((kv.first + n - ns) % n);
        std::vector<cd> d(n);
        for (u32 j = 0; j < n; j++) d[j] = kv.second[j % ns];
        auto it = out.find(o);
        if (it == out.end()) {
            out.emplace(o, std::move(d));
        } else {
            for (u32 j = 0; j < n; j++) it->second[j] += d[j];
        }
    }
    return out;
}

// the sparse CoeffToSlot's last factor: 1 on even copies of n_s slots, -i on
// odd ones; with y = f u (u repeated), y + conj(y) = 2 Re u on the even
// copies and 2 Im u on the odd ones
void times_copy_factor(Diags &M, u32 ns)
{
    for (auto &kv : M)
        for (u32 j = 0; j < kv.second.size(); j++)
            if ((j / ns) & 1) kv.second[j] *= cd(0.0, -1.0);
}

// {0: (1, i), n_s: (i, 1)} (period 2 n_s): (a, b) -> a + i b in every copy
Diags join_map(u32 ns, u32 n)
{
    std::vector<cd> p1(n), p2(n);
    for (u32 j = 0; j < n; j++) {
        const bool odd = (j / ns) & 1;
        p1[j] = odd ? cd(0.0, 1.0) : cd(1.0);
        p2[j] = odd ? cd(1.0) : cd(0.0, 1.0);
    }
    Diags out;
    out.emplace(0u, std::move(p1));
    out.emplace(ns % n, std::move(p2));
    return out;
}

u32 boot_slots(const fheon_ctx *ctx, const fheon_boot_params &p) { return p.slots ? p.slots : ctx->N / 2; }

u32 boot_depth(const fheon_boot_params &p) { return p.cts_levels + cheb_depth(p.degree) + p.doublings + p.stc_levels; }

int check_params(fheon_ctx *ctx, const fheon_boot_params *p)
{
    const u32 ns = boot_slots(ctx, *p);
    if (ns < 2 || ns > ctx->N / 2 || (ns & (ns - 1)))
        return fail(ctx, FHEON_ERR_ARG, "bootstrap: slots 0 or a power of two in [2, N/2]");
    if (p->unmasked > 1 || (p->unmasked && ns == ctx->N / 2))
        return fail(ctx, FHEON_ERR_ARG, "bootstrap: unmasked is 0 or 1, and 1 only with slots < N/2");
    u32 logn = 0;
    while ((1u << logn) < ns) logn++;
    if (!p->cts_levels || !p->stc_levels || p->cts_levels > logn || p->stc_levels > logn || !p->K ||
        p->degree < 2 || p->degree > 1023 || p->doublings > 30)
        return fail(ctx, FHEON_ERR_ARG, "bootstrap: levels in [1, log2(slots)], K >= 1, degree in [2, 1023]");
    if (boot_depth(*p) > ctx->L - 1)
        return fail(ctx, FHEON_ERR_LEVEL, "bootstrap needs %u levels above q_0, the context has %u", boot_depth(*p),
                    ctx->L - 1);
    return FHEON_OK;
}

// the scale after EvalMod's r doublings (the series keeps its input scale s),
// computed in the order the operations compute it
double evalmod_end_scale(fheon_ctx *ctx, double s, u32 lv, u32 r)
{
    for (u32 i = 0; i < r; i++) {
        s = (s * s) / (double)ctx->mod[lv - 1];
        lv--;
    }
    return s;
}

// a default layer per context, kept for the one-shot call
struct DefaultBoot {
    double scale = 0;
    fheon_layer *ly = nullptr;
};
std::map<const fheon_ctx *, DefaultBoot> g_default;
std::mutex g_default_mu;

} // namespace

namespace fheon {

static int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

void bsgs_split(const std::set<int64_t> &ks, int64_t M, u32 baby, int64_t &bs, std::set<int64_t> &ts,
                std::set<int64_t> &cs)
{
    auto split = [&](int64_t b) {
        ts.clear();
        cs.clear();
        for (int64_t k : ks) {
            const int64_t c = floordiv(k, b);
            cs.insert(c);
            ts.insert(k - c * b);
        }
    };
    bs = baby;
    if (!bs) {
        int64_t best = -1;
        for (int64_t b = 1; b <= M; b *= 2) {
            split(b);
            const int64_t cost = (int64_t)ts.size() - (int64_t)ts.count(0) + (int64_t)cs.size() - (int64_t)cs.count(0);
            if (best < 0 || cost <= best) {
                best = cost;
                bs = b;
            }
        }
    }
    split(bs);
}

std::set<int64_t> bsgs_offsets(const std::set<u32> &offsets, u32 n, u32 stride)
{
    const int64_t M = n / stride;
    std::set<int64_t> ks;
    for (u32 o : offsets) {
        int64_t k = o / stride;
        if (k > M / 2) k -= M;
        ks.insert(k);
    }
    return ks;
}

Bsgs bsgs_plan(const Diags &D, u32 n, u32 stride, u32 baby)
{
    std::set<u32> offs;
    std::map<int64_t, const std::vector<cd> *> byk;
    for (const auto &kv : D) {
        bool any = false;
        for (const cd &x : kv.second) any = any || x != cd(0.0);
        if (!any) continue;
        offs.insert(kv.first);
    }
    const std::set<int64_t> ks = bsgs_offsets(offs, n, stride);
    for (const auto &kv : D)
        if (offs.count(kv.first)) {
            const int64_t M = n / stride;
            int64_t k = kv.first / stride;
            if (k > M / 2) k -= M;
            byk[k] = &kv.second;
        }
    int64_t bs = 0;
    std::set<int64_t> ts, cs;
    bsgs_split(ks, (int64_t)(n / stride), baby, bs, ts, cs);
    Bsgs out;
    for (int64_t t : ts) out.r.push_back((int32_t)(t * stride));
    for (int64_t c : cs) {
        const int64_t G = c * bs * (int64_t)stride;
        out.s.push_back((int32_t)G);
        const u32 sh = (u32)(((G % (int64_t)n) + n) % n);
        for (int64_t t : ts) {
            auto it = byk.find(c * bs + t);
            if (it == byk.end()) {
                out.vals.emplace_back();
                continue;
            }
            // Rot_{-G}(d)[i] = d[i - G]
            std::vector<cd> v(n);
            for (u32 i = 0; i < n; i++) v[i] = (*it->second)[(i + n - sh) % n];
            out.vals.push_back(std::move(v));
        }
    }
    return out;
}

int diag_layer(fheon_ctx *ctx, const Diags &M, u32 stride, cd factor, u32 baby, u32 level, double pscale,
               fheon_layer **out)
{
    const u32 n = ctx->N / 2;
    Bsgs B = bsgs_plan(M, n, stride, baby);
    const u32 nt = (u32)B.r.size(), ng = (u32)B.s.size();
    std::vector<fheon_pt *> pts((size_t)nt * ng, nullptr);
    std::vector<double> re(n), im(n);
    int rc = FHEON_OK;
    for (size_t i = 0; i < pts.size() && !rc; i++) {
        if (B.vals[i].empty()) continue;
        for (u32 j = 0; j < n; j++) {
            const cd v = B.vals[i][j] * factor;
            re[j] = v.real();
            im[j] = v.imag();
        }
        rc = fheon_encode_plain(ctx, re.data(), im.data(), n, level, pscale, &pts[i]);
    }
    if (!rc)
        rc = fheon_linear_prepare_plain(ctx, 0, nullptr, nt, B.r.data(), ng, B.s.data(), pts.data(), nullptr, level,
                                        out);
    if (rc) {
        for (fheon_pt *p : pts) fheon_pt_destroy(p);
        return rc;
    }
    for (fheon_pt *p : pts)
        if (p) (*out)->pt_store.push_back(p);
    return FHEON_OK;
}

// x_p <- x_p + sigma_g(x_p) for every input p, the n automorphisms as one
// key-switching batch (sigma_g(x_p) lands in tmp_p)
static int add_automorph_many(fheon_ctx *ctx, fheon_ct *const *xs, fheon_ct *const *tmp, u32 n, u64 g, PlanKeep *keep)
{
    auto key = ctx->keys.find(g);
    if (key == ctx->keys.end())
        return fail(ctx, FHEON_ERR_NO_KEY, "bootstrap: no key for Galois element %llu", (unsigned long long)g);
    std::vector<KsItem> ks(n);
    int rc;
    for (u32 p = 0; p < n; p++) {
        const fheon_ct *x = xs[p];
        if ((rc = ct_reshape(ctx, tmp[p], x->level))) return rc;
        tmp[p]->scale = x->scale;
        ks[p].c0 = x->c0();
        ks[p].c1 = x->c1(ctx->N);
        ks[p].out = tmp[p]->c0();
        ks[p].key = key->second.mem.as<u64>();
        ks[p].g = g;
        ks[p].level = x->level;
        ks[p].lead = p;
    }
    if ((rc = ks_many(ctx, ks.data(), n, false, keep))) return rc;
    for (u32 p = 0; p < n; p++)
        if ((rc = fheon_add(ctx, xs[p], tmp[p], xs[p]))) return rc;
    return FHEON_OK;
}

// The sparse bootstrap of n inputs (slots [0, n_s); every step of all inputs
// as one batch): mask and repeat at the bottom, ModRaise, the trace, the
// n_s-slot CoeffToSlot, y + conj(y), one EvalMod, SlotToCoeff.
static int boot_sparse_many(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins, u32 n,
                            fheon_ct *const *outs)
{
    const u32 N = ctx->N, D = (u32)ly->coeffs.size() - 1, ns = ly->boot_ns;
    int rc;
    const u32 min_level = ly->boot_unmasked ? 1 : 2;
    for (u32 p = 0; p < n; p++) {
        if (ins[p]->level < min_level)
            return fail(ctx, FHEON_ERR_LEVEL, "sparse bootstrap: input at level %u, needs >= %u", ins[p]->level, min_level);
        if (std::fabs(ins[p]->scale - ly->in_scale) > 1e-9 * ly->in_scale)
            return fail(ctx, FHEON_ERR_SCALE, "bootstrap prepared for scale %g, got %g", ly->in_scale, ins[p]->scale);
    }
    auto conj = ctx->keys.find(2ull * N - 1);
    if (conj == ctx->keys.end()) return fail(ctx, FHEON_ERR_NO_KEY, "bootstrap: no conjugation key");
    if (ly->bsets.size() < n) ly->bsets.resize(n);
    // per input: 0 raised, 1-2 chain, 3 automorphism, 4 masked and repeated,
    // 5-6 doubling ping-pong, 7 the input at level 2
    for (u32 p = 0; p < n; p++) {
        auto &w = ly->bsets[p].w;
        if (w.size() < 8) w.resize(8, nullptr);
        for (fheon_ct *&c : w)
            if (!c && (rc = fheon_ct_create(ctx, 1, 1.0, &c))) return rc;
    }
    auto W = [&](u32 p, u32 i) { return ly->bsets[p].w[i]; };
    std::vector<fheon_ct *> xs(n), tmp(n), dsts(n);
    for (u32 p = 0; p < n; p++) {
        if (ly->boot_unmasked) {
            if ((rc = fheon_drop_level(ctx, ins[p], 1, W(p, 4)))) return rc;
        } else {
            if ((rc = fheon_drop_level(ctx, ins[p], 2, W(p, 7)))) return rc;
            if ((rc = fheon_mul_plain(ctx, W(p, 7), ly->boot_mask, W(p, 4)))) return rc;
            if ((rc = fheon_rescale(ctx, W(p, 4), W(p, 4)))) return rc;
        }
        xs[p] = W(p, 4);
        tmp[p] = W(p, 3);
    }
    // the copies' automorphisms: Rot_{n_s}, Rot_{2 n_s}, ...
    std::vector<u64> gs;
    for (u32 st = ns; st < N / 2; st <<= 1) gs.push_back(fheon_galois_elt(ctx, (int32_t)st));
    for (u64 g : gs)
        if ((rc = add_automorph_many(ctx, xs.data(), tmp.data(), n, g, ly->collect))) return rc;
    for (u32 p = 0; p < n; p++) {
        if ((rc = mod_raise_ct(ctx, W(p, 4), W(p, 0)))) return rc;
        W(p, 0)->scale = (double)ctx->mod[0];
        xs[p] = W(p, 0);
    }
    {
        Range range("Trace");
        for (u64 g : gs)
            if ((rc = add_automorph_many(ctx, xs.data(), tmp.data(), n, g, ly->collect))) return rc;
    }
    std::vector<const fheon_ct *> cx(xs.begin(), xs.end());
    auto sub_apply = [&](const fheon_layer *sub, fheon_ct *const *to) {
        sub->collect = ly->collect;
        const int r = fheon_layer_apply_batch(ctx, sub, cx.data(), n, to);
        sub->collect = nullptr;
        return r;
    };
    {
        Range range("CoeffToSlot");
        for (u32 i = 0; i < ly->ncts; i++) {
            for (u32 p = 0; p < n; p++) dsts[p] = W(p, 1 + (i & 1));
            if ((rc = sub_apply(ly->subs[i], dsts.data()))) return rc;
            for (u32 p = 0; p < n; p++) cx[p] = dsts[p];
        }
    }
    Range phase("EvalMod");
    // y + conj(y): the low coefficients in the even copies, the high ones in
    // the odd copies -- EvalMod's one input
    std::vector<KsItem> ks(n);
    for (u32 p = 0; p < n; p++) {
        const fheon_ct *x = cx[p];
        if ((rc = ct_reshape(ctx, W(p, 3), x->level))) return rc;
        W(p, 3)->scale = x->scale;
        ks[p].c0 = x->c0();
        ks[p].c1 = x->c1(N);
        ks[p].out = W(p, 3)->c0();
        ks[p].key = conj->second.mem.as<u64>();
        ks[p].g = 2ull * N - 1;
        ks[p].level = x->level;
        ks[p].lead = p;
    }
    if ((rc = ks_many(ctx, ks.data(), n, false, ly->collect))) return rc;
    std::vector<std::vector<fheon_ct *> *> works(n);
    std::vector<fheon_ct *> a(n), b(n);
    for (u32 p = 0; p < n; p++) {
        const fheon_ct *x = cx[p];
        auto &bs = ly->bsets[p];
        if ((rc = cheb_work(ctx, bs.re, D, x->level, x->scale))) return rc;
        if ((rc = fheon_add(ctx, x, W(p, 3), bs.re[1]))) return rc;
        works[p] = &bs.re;
        a[p] = W(p, 5);
        b[p] = W(p, 6);
    }
    if ((rc = cheb_series_many(ctx, ly->coeffs, works.data(), n, a.data(), ly->collect))) return rc;
    std::vector<RelinItem> it(n);
    for (u32 i = 0; i < ly->boot_r; i++) {
        for (u32 k = 0; k < n; k++) it[k] = RelinItem{a[k], a[k], a[k]->level, true, b[k]};
        if ((rc = mul_relin_many(ctx, it.data(), n, ly->collect))) return rc;
        for (u32 k = 0; k < n; k++) {
            if ((rc = fheon_rescale(ctx, b[k], b[k]))) return rc;
            if ((rc = fheon_add_const(ctx, b[k], -1.0, b[k]))) return rc;
            std::swap(a[k], b[k]);
        }
    }
    for (u32 p = 0; p < n; p++) cx[p] = a[p];
    phase.next("SlotToCoeff");
    const u32 nst = (u32)ly->subs.size() - ly->ncts;
    for (u32 i = 0; i < nst; i++) {
        for (u32 p = 0; p < n; p++) dsts[p] = i + 1 == nst ? outs[p] : W(p, 1 + (i & 1));
        if ((rc = sub_apply(ly->subs[ly->ncts + i], dsts.data()))) return rc;
        for (u32 p = 0; p < n; p++) cx[p] = dsts[p];
    }
    return FHEON_OK;
}

int boot_apply(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *out)
{
    if (ly->boot_ns) return boot_sparse_many(ctx, ly, &in, 1, &out);
    if (in->level < 1) return fail(ctx, FHEON_ERR_LEVEL, "bootstrap: empty ciphertext");
    if (std::fabs(in->scale - ly->in_scale) > 1e-9 * ly->in_scale)
        return fail(ctx, FHEON_ERR_SCALE, "bootstrap prepared for scale %g, got %g", ly->in_scale, in->scale);
    const u32 N = ctx->N, D = (u32)ly->coeffs.size() - 1;
    int rc;
    // working ciphertexts: 0 raised, 1-2 chain, 3 conjugate, 4 difference,
    // 5-6 doubling ping-pong (re), 7-8 (im), 9 product
    if (ly->work.size() < 10) ly->work.resize(10, nullptr);
    for (fheon_ct *&c : ly->work)
        if (!c && (rc = fheon_ct_create(ctx, 1, 1.0, &c))) return rc;
    fheon_ct **w = ly->work.data();
    if ((rc = mod_raise_ct(ctx, in, w[0]))) return rc;
    w[0]->scale = (double)ctx->mod[0];
    const fheon_ct *x = w[0];
    // the levels' batched rotations read device plans: while this layer is
    // captured into a graph, the graph keeps them (the levels report to the
    // same collector)
    auto sub_apply = [&](const fheon_layer *sub, const fheon_ct *a, fheon_ct *b) {
        sub->collect = ly->collect;
        const int r = fheon_layer_apply(ctx, sub, a, b);
        sub->collect = nullptr;
        return r;
    };
    {
        Range range("CoeffToSlot");
        for (u32 i = 0; i < ly->ncts; i++) {
            fheon_ct *dst = w[1 + (i & 1)];
            if ((rc = sub_apply(ly->subs[i], x, dst))) return rc;
            x = dst;
        }
    }
    Range phase("EvalMod");
    // real and imaginary parts: T_1 of each part's series
    const u32 lv = x->level;
    if ((rc = cheb_work(ctx, ly->rot, D, lv, x->scale))) return rc;
    if ((rc = cheb_work(ctx, ly->cheb2, D, lv, x->scale))) return rc;
    if ((rc = fheon_rotate_galois(ctx, x, 2ull * N - 1, w[3]))) return rc;
    if ((rc = fheon_add(ctx, x, w[3], ly->rot[1]))) return rc;
    if ((rc = fheon_mul_int(ctx, x, -1, w[4]))) return rc;
    if ((rc = fheon_add(ctx, w[3], w[4], w[4]))) return rc;
    if ((rc = fheon_mul_plain(ctx, w[4], ly->mono[0], ly->cheb2[1]))) return rc;
    // EvalMod on both parts in lockstep: every product of a step is one batch
    std::vector<fheon_ct *> *works[2] = {&ly->rot, &ly->cheb2};
    fheon_ct *a[2] = {w[5], w[7]}, *b[2] = {w[6], w[8]};
    if ((rc = cheb_series_many(ctx, ly->coeffs, works, 2, a, ly->collect))) return rc;
    for (u32 i = 0; i < ly->boot_r; i++) {
        // 2 c^2 - 1: the doubled product rescaled, then -1 at the new scale
        RelinItem it[2] = {RelinItem{a[0], a[0], a[0]->level, true, b[0]}, RelinItem{a[1], a[1], a[1]->level, true, b[1]}};
        if ((rc = mul_relin_many(ctx, it, 2, ly->collect))) return rc;
        for (int k = 0; k < 2; k++) {
            if ((rc = fheon_rescale(ctx, b[k], b[k]))) return rc;
            if ((rc = fheon_add_const(ctx, b[k], -1.0, b[k]))) return rc;
            std::swap(a[k], b[k]);
        }
    }
    fheon_ct *part[2] = {a[0], a[1]};
    if ((rc = fheon_mul_plain(ctx, part[1], ly->mono[1], w[9]))) return rc;
    if ((rc = fheon_add(ctx, part[0], w[9], w[9]))) return rc;
    phase.next("SlotToCoeff");
    x = w[9];
    const u32 nst = (u32)ly->subs.size() - ly->ncts;
    for (u32 i = 0; i < nst; i++) {
        fheon_ct *dst = i + 1 == nst ? out : w[1 + (i & 1)];
        if ((rc = sub_apply(ly->subs[ly->ncts + i], x, dst))) return rc;
        x = dst;
    }
    return FHEON_OK;
}

int boot_apply_many(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins, u32 n, fheon_ct *const *outs)
{
    if (ly->boot_ns) return boot_sparse_many(ctx, ly, ins, n, outs);
    const u32 N = ctx->N, D = (u32)ly->coeffs.size() - 1;
    int rc;
    for (u32 p = 0; p < n; p++) {
        if (ins[p]->level < 1) return fail(ctx, FHEON_ERR_LEVEL, "bootstrap: empty ciphertext");
        if (std::fabs(ins[p]->scale - ly->in_scale) > 1e-9 * ly->in_scale)
            return fail(ctx, FHEON_ERR_SCALE, "bootstrap prepared for scale %g, got %g", ly->in_scale, ins[p]->scale);
    }
    auto conj = ctx->keys.find(2ull * N - 1);
    if (conj == ctx->keys.end()) return fail(ctx, FHEON_ERR_NO_KEY, "bootstrap: no conjugation key");
    if (ly->bsets.size() < n) ly->bsets.resize(n);
    // per input: 0 raised, 1-2 chain, 3 conjugate, 4 difference, 5-8 doubling
    // ping-pong (re, im), 9 recombined
    for (u32 p = 0; p < n; p++) {
        auto &w = ly->bsets[p].w;
        if (w.size() < 10) w.resize(10, nullptr);
        for (fheon_ct *&c : w)
            if (!c && (rc = fheon_ct_create(ctx, 1, 1.0, &c))) return rc;
    }
    auto W = [&](u32 p, u32 i) { return ly->bsets[p].w[i]; };
    std::vector<const fheon_ct *> xs(n);
    std::vector<fheon_ct *> dsts(n);
    for (u32 p = 0; p < n; p++) {
        if ((rc = mod_raise_ct(ctx, ins[p], W(p, 0)))) return rc;
        W(p, 0)->scale = (double)ctx->mod[0];
        xs[p] = W(p, 0);
    }
    auto sub_apply = [&](const fheon_layer *sub, fheon_ct *const *to) {
        sub->collect = ly->collect;
        const int r = fheon_layer_apply_batch(ctx, sub, xs.data(), n, to);
        sub->collect = nullptr;
        return r;
    };
    {
        Range range("CoeffToSlot");
        for (u32 i = 0; i < ly->ncts; i++) {
            for (u32 p = 0; p < n; p++) dsts[p] = W(p, 1 + (i & 1));
            if ((rc = sub_apply(ly->subs[i], dsts.data()))) return rc;
            for (u32 p = 0; p < n; p++) xs[p] = dsts[p];
        }
    }
    Range phase("EvalMod");
    // the conjugates of every input as one key-switching batch
    std::vector<KsItem> ks(n);
    for (u32 p = 0; p < n; p++) {
        const fheon_ct *x = xs[p];
        if ((rc = ct_reshape(ctx, W(p, 3), x->level))) return rc;
        W(p, 3)->scale = x->scale;
        ks[p].c0 = x->c0();
        ks[p].c1 = x->c1(N);
        ks[p].out = W(p, 3)->c0();
        ks[p].key = conj->second.mem.as<u64>();
        ks[p].g = 2ull * N - 1;
        ks[p].level = x->level;
        ks[p].lead = p;
    }
    if ((rc = ks_many(ctx, ks.data(), n, false, ly->collect))) return rc;
    std::vector<std::vector<fheon_ct *> *> works(2 * n);
    std::vector<fheon_ct *> a(2 * n), b(2 * n);
    for (u32 p = 0; p < n; p++) {
        const fheon_ct *x = xs[p];
        auto &bs = ly->bsets[p];
        if ((rc = cheb_work(ctx, bs.re, D, x->level, x->scale))) return rc;
        if ((rc = cheb_work(ctx, bs.im, D, x->level, x->scale))) return rc;
        if ((rc = fheon_add(ctx, x, W(p, 3), bs.re[1]))) return rc;
        if ((rc = fheon_mul_int(ctx, x, -1, W(p, 4)))) return rc;
        if ((rc = fheon_add(ctx, W(p, 3), W(p, 4), W(p, 4)))) return rc;
        if ((rc = fheon_mul_plain(ctx, W(p, 4), ly->mono[0], bs.im[1]))) return rc;
        works[2 * p] = &bs.re;
        works[2 * p + 1] = &bs.im;
        a[2 * p] = W(p, 5);
        a[2 * p + 1] = W(p, 7);
        b[2 * p] = W(p, 6);
        b[2 * p + 1] = W(p, 8);
    }
    if ((rc = cheb_series_many(ctx, ly->coeffs, works.data(), 2 * n, a.data(), ly->collect))) return rc;
    std::vector<RelinItem> it(2 * n);
    for (u32 i = 0; i < ly->boot_r; i++) {
        for (u32 k = 0; k < 2 * n; k++) it[k] = RelinItem{a[k], a[k], a[k]->level, true, b[k]};
        if ((rc = mul_relin_many(ctx, it.data(), 2 * n, ly->collect))) return rc;
        for (u32 k = 0; k < 2 * n; k++) {
            if ((rc = fheon_rescale(ctx, b[k], b[k]))) return rc;
            if ((rc = fheon_add_const(ctx, b[k], -1.0, b[k]))) return rc;
            std::swap(a[k], b[k]);
        }
    }
    for (u32 p = 0; p < n; p++) {
        if ((rc = fheon_mul_plain(ctx, a[2 * p + 1], ly->mono[1], W(p, 9)))) return rc;
        if ((rc = fheon_add(ctx, a[2 * p], W(p, 9), W(p, 9)))) return rc;
        xs[p] = W(p, 9);
    }
    phase.next("SlotToCoeff");
    const u32 nst = (u32)ly->subs.size() - ly->ncts;
    for (u32 i = 0; i < nst; i++) {
        for (u32 p = 0; p < n; p++) dsts[p] = i + 1 == nst ? outs[p] : W(p, 1 + (i & 1));
        if ((rc = sub_apply(ly->subs[ly->ncts + i], dsts.data()))) return rc;
        for (u32 p = 0; p < n; p++) xs[p] = dsts[p];
    }
    return FHEON_OK;
}

} // namespace fheon

extern "C" {

int fheon_boot_params_default(const fheon_ctx *ctx, fheon_boot_params *p)
{
    if (!ctx || !p) return FHEON_ERR_ARG;
    p->cts_levels = 3;
    p->stc_levels = 3;
    // |t / q_0| for a uniform ternary secret: a coefficient of c_1 s sums about
    // 2N/3 terms uniform in [-q_0/2, q_0/2), standard deviation ~ sqrt(N/18);
    // K = the power of two at or above 8 of those
    const double x = 8.0 * std::sqrt((double)ctx->N / 18.0);
    u32 K = 1;
    while ((double)K < x) K *= 2;
    p->K = K;
    u32 r = 0;
    while ((1u << r) < K) r++;
    p->doublings = r;
    p->degree = 27;
    p->baby = 0;
    p->slots = 0;
    p->unmasked = 0;
    return FHEON_OK;
}

int fheon_evalmod_coeffs(uint32_t K, uint32_t doublings, uint32_t degree, double *out)
{
    if (!out || !K || degree < 1 || degree > 1023 || doublings > 30) return FHEON_ERR_ARG;
    const u32 D = degree;
    for (u32 d = 0; d <= D; d++) {
        double sum = 0.0;
        for (u32 k = 0; k <= D; k++) {
            const double th = M_PI * ((double)k + 0.5) / (double)(D + 1);
            const double z = std::cos(th);
            const double f = std::cos((2.0 * M_PI) * ((double)K * z - 0.25) / std::ldexp(1.0, (int)doublings));
            sum += f * std::cos((double)d * th);
        }
        out[d] = sum * 2.0 / (double)(D + 1);
    }
    out[0] *= 0.5;
    return FHEON_OK;
}

int fheon_bootstrap_compose(fheon_ctx *ctx, const fheon_boot_params *p, const fheon_layer *const *cts,
                            const fheon_layer *const *stc, const double *coeffs, double in_scale, fheon_layer **out)
{
    if (!ctx || !p || !cts || !stc || !coeffs || !out || !(in_scale > 0)) return FHEON_ERR_ARG;
    int rc = check_params(ctx, p);
    if (rc) return rc;
    const u32 L = ctx->L;
    u32 lv = L;
    for (u32 i = 0; i < p->cts_levels + p->stc_levels; i++) {
        const fheon_layer *s = i < p->cts_levels ? cts[i] : stc[i - p->cts_levels];
        if (!s || s->kind != LAYER_LINEAR || !s->fold.empty() || s->bias)
            return fail(ctx, FHEON_ERR_ARG, "bootstrap: level %u is not a rotation-sum layer", i);
        if (i == p->cts_levels) lv -= cheb_depth(p->degree) + p->doublings;
        if (s->level != lv) return fail(ctx, FHEON_ERR_LEVEL, "bootstrap: level %u at %u, expected %u", i, s->level, lv);
        lv--;
    }
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_BOOT;
    ly->level = L;
    ly->ncts = p->cts_levels;
    for (u32 i = 0; i < p->cts_levels; i++) ly->subs.push_back(const_cast<fheon_layer *>(cts[i]));
    for (u32 i = 0; i < p->stc_levels; i++) ly->subs.push_back(const_cast<fheon_layer *>(stc[i]));
    ly->coeffs.assign(coeffs, coeffs + p->degree + 1);
    ly->boot_K = p->K;
    ly->boot_r = p->doublings;
    ly->in_scale = in_scale;
    ly->out_level = lv;
    const u32 n = ctx->N / 2, ns = boot_slots(ctx, *p);
    if (ns < n && p->unmasked) {
        ly->boot_ns = ns;
        ly->nslots = n;
        ly->boot_unmasked = true;
        *out = ly.release();
        return FHEON_OK;
    }
    if (ns < n) {
        // the input mask: 1 in slots [0, n_s), at level 2 and scale q_1, the
        // prime its rescale drops
        if (L < 2) return fail(ctx, FHEON_ERR_LEVEL, "sparse bootstrap: the context needs 2 primes");
        std::vector<double> re(n, 0.0), im(n, 0.0);
        for (u32 j = 0; j < ns; j++) re[j] = 1.0;
        fheon_pt *mask = nullptr;
        if ((rc = fheon_encode_plain(ctx, re.data(), im.data(), n, 2, (double)ctx->mod[1], &mask))) return rc;
        ly->boot_ns = ns;
        ly->nslots = n;
        ly->boot_mask = mask;
        ly->own_boot_mask = true;
        *out = ly.release();
        return FHEON_OK;
    }
    // X^(N/2) (the constant i in every slot, scale 1) where im is formed and
    // where the parts are recombined
    std::vector<int64_t> mono(ctx->N, 0);
    mono[ctx->N / 2] = 1;
    const u32 l0 = L - p->cts_levels, l1 = l0 - cheb_depth(p->degree) - p->doublings;
    if ((rc = fheon_plain_from_coeffs(ctx, mono.data(), l0, 1.0, &ly->mono[0]))) return rc;
    if ((rc = fheon_plain_from_coeffs(ctx, mono.data(), l1, 1.0, &ly->mono[1]))) return rc;
    *out = ly.release();
    return FHEON_OK;
}

int fheon_bootstrap_prepare(fheon_ctx *ctx, const fheon_boot_params *p_, double in_scale, fheon_layer **out)
{
    if (!ctx || !out || !(in_scale > 0)) return FHEON_ERR_ARG;
    fheon_boot_params p;
    if (p_) {
        p = *p_;
    } else {
        fheon_boot_params_default(ctx, &p);
    }
    int rc = check_params(ctx, &p);
    if (rc) return rc;
    const u32 L = ctx->L, n = ctx->N / 2;
    std::vector<double> coeffs(p.degree + 1);
    if ((rc = fheon_evalmod_coeffs(p.K, p.doublings, p.degree, coeffs.data()))) return rc;
    std::vector<fheon_layer *> subs;
    auto cleanup = [&]() {
        for (fheon_layer *l : subs) delete l;
    };
    u32 lv = L;
    double s = (double)ctx->mod[0];
    const double q0 = (double)ctx->mod[0];
    // CoeffToSlot: 1/(2K) and the change of scale q_0 -> Delta_b in the first
    // level.  Sparse: the n_s-slot transform in every copy, 1/copies in the
    // first level (the trace summed the copies), the copy factor in the last
    const u32 ns = boot_slots(ctx, p), copies = n / ns;
    const double delta_b = (double)ctx->mod[L - p.cts_levels - 1];
    auto cl = merged_levels(ns, p.cts_levels, true);
    for (u32 i = 0; i < p.cts_levels; i++) {
        const double q = (double)ctx->mod[lv - 1];
        const double ps = i == 0 ? q * (delta_b / q0) : q;
        fheon_layer *l = nullptr;
        Diags M = ns < n ? replicate(cl[i].M, ns, n) : std::move(cl[i].M);
        if (ns < n && i + 1 == p.cts_levels) times_copy_factor(M, ns);
        const cd f(i == 0 ? 1.0 / (2.0 * (double)p.K * (double)copies) : 1.0);
        if ((rc = diag_layer(ctx, M, cl[i].stride, f, p.baby, lv, ps, &l))) {
            cleanup();
            return rc;
        }
        subs.push_back(l);
        s = (s * ps) / q;
        lv--;
    }
    lv -= cheb_depth(p.degree);
    s = evalmod_end_scale(ctx, s, lv, p.doublings);
    lv -= p.doublings;
    // SlotToCoeff: q_0 / (2 pi Delta_in) in the first level, the change of
    // scale onto Delta_in in the last
    // (sparse: the n_s-slot transform in every copy, the join map first)
    auto sl = merged_levels(ns, p.stc_levels, false);
    for (u32 i = 0; i < p.stc_levels; i++) {
        const double q = (double)ctx->mod[lv - 1];
        const double ps = i + 1 == p.stc_levels ? q * (in_scale / s) : q;
        fheon_layer *l = nullptr;
        const cd f(i == 0 ? q0 / (2.0 * M_PI * in_scale) : 1.0);
        Diags M = ns < n ? replicate(sl[i].M, ns, n) : std::move(sl[i].M);
        u32 stride = sl[i].stride;
        if (ns < n && i == 0) {
            M = compose(M, join_map(ns, n), n);
            stride = 1;
        }
        if ((rc = diag_layer(ctx, M, stride, f, p.baby, lv, ps, &l))) {
            cleanup();
            return rc;
        }
        subs.push_back(l);
        s = (s * ps) / q;
        lv--;
    }
    rc = fheon_bootstrap_compose(ctx, &p, subs.data(), subs.data() + p.cts_levels, coeffs.data(), in_scale, out);
    if (rc) {
        cleanup();
        return rc;
    }
    (*out)->own_subs = true;
    (*out)->out_scale = s;
    return FHEON_OK;
}

int fheon_bootstrap_set_mask(fheon_ctx *ctx, fheon_layer *ly, const fheon_pt *mask)
{
    if (!ctx || !ly || !mask || ly->kind != LAYER_BOOT) return FHEON_ERR_ARG;
    if (!ly->boot_ns || ly->boot_unmasked) return fail(ctx, FHEON_ERR_ARG, "set_mask: not a masked sparse bootstrap");
    if (mask->level < 2) return fail(ctx, FHEON_ERR_ARG, "set_mask: the mask must be at level >= 2");
    if (ly->own_boot_mask) fheon_pt_destroy(const_cast<fheon_pt *>(ly->boot_mask));
    ly->boot_mask = mask;
    ly->own_boot_mask = false;
    return FHEON_OK;
}

int fheon_bootstrap_keygen(fheon_ctx *ctx, const fheon_sk *sk, const fheon_layer *ly)
{
    if (!ctx || !sk || !ly || ly->kind != LAYER_BOOT) return FHEON_ERR_ARG;
    u32 n = 0;
    int rc = fheon_layer_rotation_steps(ly, nullptr, &n);
    if (rc) return rc;
    std::vector<int32_t> st(n);
    if ((rc = fheon_layer_rotation_steps(ly, st.data(), &n))) return rc;
    if ((rc = fheon_rotkeygen(ctx, sk, st.data(), n))) return rc;
    const uint64_t conj = 2ull * ctx->N - 1;
    if ((rc = fheon_galois_keygen(ctx, sk, &conj, 1))) return rc;
    return fheon_relinkeygen(ctx, sk);
}

int fheon_bootstrap_info(const fheon_layer *ly, uint32_t *out_level, double *out_scale)
{
    if (!ly || ly->kind != LAYER_BOOT) return FHEON_ERR_ARG;
    if (out_level) *out_level = ly->out_level;
    if (out_scale) *out_scale = ly->out_scale;
    return FHEON_OK;
}

int fheon_mod_raise(fheon_ctx *ctx, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !in || !out || in->level < 1) return FHEON_ERR_ARG;
    int rc = mod_raise_ct(ctx, in, out);
    if (rc) return rc;
    out->scale = in->scale;
    return FHEON_OK;
}

int fheon_bootstrap(fheon_ctx *ctx, const fheon_ct *ct, fheon_ct *out)
{
    if (!ctx || !ct || !out) return FHEON_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_default_mu);
    DefaultBoot &d = g_default[ctx];
    if (!d.ly || std::fabs(d.scale - ct->scale) > 1e-9 * ct->scale) {
        if (d.ly) {
            cudaStreamSynchronize(ctx->stream);
            delete d.ly;
            d.ly = nullptr;
        }
        int rc = fheon_bootstrap_prepare(ctx, nullptr, ct->scale, &d.ly);
        if (rc) {
            g_default.erase(ctx);
            return rc;
        }
        d.scale = ct->scale;
    }
    return fheon_layer_apply(ctx, d.ly, ct, out);
}

} // extern "C"

namespace fheon {
// the one-shot call's cached layer of a context that is going away
void boot_release(const fheon_ctx *ctx)
{
    std::lock_guard<std::mutex> lk(g_default_mu);
    auto it = g_default.find(ctx);
    if (it == g_default.end()) return;
    delete it->second.ly;
    g_default.erase(it);
}
} // namespace fheon
