// linear.cu -- the linear layers of an encrypted CNN on a packed feature map
// (fheon_map): convolution (paper Sec. 5.1 equation; any zero padding and
// stride, C input and F output channels; the stride selects the output
// positions the weights are placed at), average pooling (Sec. 5.4: the window sum
// times a 1/k^2 mask that also does the striding, the outputs staying at
// stride-aligned slots) and the fully connected layer (Sec. 5.5: one product
// per output neuron, the sum of its slots, a one-hot placement).
//
// Rotation-sum layer (conv, pooling):
//   out = sum_g Rot_{s_g}( rescale( sum_t Rot_{r_t}(in) * P_{g,t} ) ) (+ bias)
// The tap rotations r_t are hoisted from the input (one raising of c1); each
// group's products are summed in one pass (fheon_mac_plain) and rescaled once;
// the group sums move by one batched rotation and are added.  A conv from C to
// F channels sums, for every block shift delta = f - c, the products that in
// the block of input channel c hold K[f, c, x, y] at every output position
// whose tap source (i + x - pad, j + y - pad) lies inside the input, moved to
// block f by Rot_{-delta*block}.  Tap (x, y) reads the input at
// r = dil*((x - pad)*grid + (y - pad)).  The shifts go by baby steps and giant
// steps: delta = a + B*b, Rot_{-delta*block}(P * Rot_r(x)) =
// Rot_{-B*b*block}(Rot_{-a*block}(P) * Rot_{r - a*block}(x)), so the layer's
// taps are the B*k^2 hoisted rotations r - a*block and its groups the giant
// steps b, with B (conv_baby) the fewest rotations when a plain rotation costs
// two hoisted ones: B k^2 - 1 + 2 ceil((C + F - 1)/B).
//
// FC: t_k = rescale(in * W_k) (W_k: row k of the weights at the input's
// slots); every t_k through the rotate-and-add slot sum (steps 1, 2, 4, ...,
// N/4: the total lands in every slot); out = rescale(sum_k t_k * E_k), E_k one
// at slot k.  The output map is the compact vector of the m neurons.
#include <algorithm>
#include <cmath>
#include <memory>
#include <set>
#include <vector>

#include "layer.h"

using namespace fheon;

namespace {

u32 map_slot(const fheon_map &m, u32 c, u32 i, u32 j) { return c * m.block + m.dil * (i * m.grid + j); }

bool map_ok(const fheon_ctx *ctx, const fheon_map &m)
{
    if (!m.C || !m.H || !m.W || !m.dil || m.grid < m.W || !m.block) return false;
    if ((u64)m.dil * ((u64)(m.H - 1) * m.grid + (m.W - 1)) >= m.block) return false;
    return (u64)m.C * m.block <= ctx->N / 2;
}

int ensure_cts(fheon_ctx *ctx, std::vector<fheon_ct *> &v, size_t n, u32 level, double scale)
{
    if (v.size() < n) v.resize(n, nullptr);
    for (size_t i = 0; i < n; i++)
        if (!v[i]) {
            int rc = fheon_ct_create(ctx, level, scale, &v[i]);
            if (rc) return rc;
        }
    return FHEON_OK;
}

// the layer's own plaintext of `v` at `level` and `scale`; null when v is all zero
int own_plain(fheon_ctx *ctx, fheon_layer *ly, const std::vector<double> &v, u32 level, double scale,
              fheon_pt **out)
{
    *out = nullptr;
    bool any = false;
    for (double x : v) any = any || x != 0.0;
    if (!any) return FHEON_OK;
    int rc = fheon_encode_plain(ctx, v.data(), nullptr, (uint32_t)v.size(), level, scale, out);
    if (rc) return rc;
    ly->pt_store.push_back(*out);
    return FHEON_OK;
}

// groups g0 .. g0 + gn - 1 of a rotation-sum layer on one input: w[gg] = sum_t
// tap_t * P_{g0+gg, t} (tap_t = Rot_{r_t}(in): rot[idx[t]], or in itself for
// r_t = 0), all in one pass over the taps any of them uses (k_mac_groups: a
// tap crosses HBM about once per MACG_BLOCK_GROUPS groups); more taps than it
// takes, or products of different scales, go group by group through
// fheon_mac_plain (which reports the error)
int group_sums(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *const *rot,
               const std::vector<int> &idx, u32 g0, u32 gn, fheon_ct *const *w)
{
    const u32 nt = (u32)ly->r.size();
    std::vector<u32> used;
    for (u32 t = 0; t < nt; t++)
        for (u32 gg = 0; gg < gn; gg++)
            if (ly->pts[(size_t)(g0 + gg) * nt + t]) {
                used.push_back(t);
                break;
            }
    auto tap = [&](u32 t) -> const fheon_ct * { return idx[t] < 0 ? in : rot[idx[t]]; };
    const u32 l = in->level;
    bool grouped = !used.empty() && used.size() <= MACG_TAPS && gn <= MACG_GROUPS;
    std::vector<double> sc(gn, 0.0);
    for (u32 gg = 0; gg < gn && grouped; gg++) {
        for (u32 t : used) {
            const fheon_pt *p = ly->pts[(size_t)(g0 + gg) * nt + t];
            if (!p) continue;
            const double x = tap(t)->scale * p->scale;
            if (tap(t)->level != l || p->level < l || (sc[gg] != 0.0 && std::fabs(x - sc[gg]) > 1e-9 * sc[gg]))
                grouped = false;
            if (sc[gg] == 0.0) sc[gg] = x;
        }
        grouped = grouped && sc[gg] != 0.0;
    }
    int rc;
    if (grouped) {
        std::vector<const u64 *> cts, pts;
        std::vector<u64 *> outs;
        for (u32 t : used) cts.push_back(tap(t)->c0());
        for (u32 gg = 0; gg < gn; gg++) {
            for (u32 t : used) {
                const fheon_pt *p = ly->pts[(size_t)(g0 + gg) * nt + t];
                pts.push_back(p ? p->m.as<u64>() : nullptr);
            }
            if ((rc = ct_reshape(ctx, w[gg], l))) return rc;
            w[gg]->scale = sc[gg];
            outs.push_back(w[gg]->c0());
        }
        FHEON_CUDA(ctx, k_mac_groups(ctx, cts.data(), (u32)cts.size(), pts.data(), gn, outs.data(), l));
        return FHEON_OK;
    }
    std::vector<const fheon_ct *> srcs;
    std::vector<const fheon_pt *> ps;
    for (u32 gg = 0; gg < gn; gg++) {
        srcs.clear();
        ps.clear();
        for (u32 t = 0; t < nt; t++) {
            const fheon_pt *p = ly->pts[(size_t)(g0 + gg) * nt + t];
            if (!p) continue;
            srcs.push_back(tap(t));
            ps.push_back(p);
        }
        if ((rc = fheon_mac_plain(ctx, srcs.data(), ps.data(), (u32)srcs.size(), w[gg]))) return rc;
    }
    return FHEON_OK;
}

// n inputs at once: every input's tap rotations in one hoisted plan (grouped by
// input), the group shifts of every input in one plain batch per chunk of
// groups; the result of each input is the one it gets alone
int linear_apply(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins_, u32 n, fheon_ct *const *outs)
{
    const u32 nt = (u32)ly->r.size(), ng = (u32)ly->s.size(), nf = (u32)ly->fold.size();
    std::vector<const fheon_ct *> ins(ins_, ins_ + n);
    int rc;
    if (nf) {
        // fold: x' = sum_c Rot_{fold[c]}(x), the rotations hoisted from x
        if ((rc = ensure_cts(ctx, ly->fwork, (size_t)n * (nf + 1), ins[0]->level, ins[0]->scale))) return rc;
        std::vector<fheon_rot_item> fi;
        for (u32 i = 0; i < n; i++)
            for (u32 c = 0; c < nf; c++)
                if (ly->fold[c]) fi.push_back(fheon_rot_item{ins[i], ly->fwork[(size_t)i * (nf + 1) + c], ly->fold[c]});
        if ((rc = rotate_many(ctx, fi.data(), (u32)fi.size(), true, ly->collect))) return rc;
        for (u32 i = 0; i < n; i++) {
            fheon_ct *const *fw = ly->fwork.data() + (size_t)i * (nf + 1);
            auto part = [&](u32 c) -> const fheon_ct * { return ly->fold[c] ? fw[c] : ins[i]; };
            fheon_ct *sum = fw[nf];
            if (nf == 1) {
                if ((rc = fheon_drop_level(ctx, part(0), part(0)->level, sum))) return rc;
            } else {
                if ((rc = fheon_add(ctx, part(0), part(1), sum))) return rc;
                for (u32 c = 2; c < nf; c++)
                    if ((rc = fheon_add(ctx, sum, part(c), sum))) return rc;
            }
            ins[i] = sum;
        }
    }
    std::vector<int32_t> steps;
    std::vector<int> idx(nt, -1);
    for (u32 t = 0; t < nt; t++)
        if (ly->r[t] != 0) {
            idx[t] = (int)steps.size();
            steps.push_back(ly->r[t]);
        }
    const u32 ns = (u32)steps.size();
    // the groups go in chunks of GC: each chunk's sums are formed, moved by one
    // batched rotation and added to the output in order, so the working set
    // is bounded by the chunk and not by the layer's group count
    constexpr u32 GC_MAX = 32;
    const u32 GC = std::min(ng, GC_MAX);
    if ((rc = ensure_cts(ctx, ly->rot, (size_t)n * ns, ins[0]->level, ins[0]->scale))) return rc;
    if ((rc = ensure_cts(ctx, ly->work, (size_t)n * 2 * GC, ins[0]->level, ins[0]->scale))) return rc;
    std::vector<fheon_rot_item> items;
    for (u32 i = 0; i < n; i++)
        for (u32 k = 0; k < ns; k++) items.push_back(fheon_rot_item{ins[i], ly->rot[(size_t)i * ns + k], steps[k]});
    if ((rc = rotate_many(ctx, items.data(), (u32)items.size(), true, ly->collect))) return rc;
    std::vector<fheon_rot_item> moves;
    for (u32 g0 = 0; g0 < ng; g0 += GC) {
        const u32 gn = std::min(GC, ng - g0);
        moves.clear();
        for (u32 i = 0; i < n; i++) {
            fheon_ct *const *w = ly->work.data() + (size_t)i * 2 * GC;
            if ((rc = group_sums(ctx, ly, ins[i], ly->rot.data() + (size_t)i * ns, idx, g0, gn, w))) return rc;
            for (u32 gg = 0; gg < gn; gg++) {
                const u32 g = g0 + gg;
                if ((rc = fheon_rescale(ctx, w[gg], w[gg]))) return rc;
                if (ly->s[g] != 0) moves.push_back(fheon_rot_item{w[gg], w[GC + gg], ly->s[g]});
            }
        }
        if ((rc = rotate_many(ctx, moves.data(), (u32)moves.size(), false, ly->collect))) return rc;
        for (u32 i = 0; i < n; i++) {
            fheon_ct *const *w = ly->work.data() + (size_t)i * 2 * GC;
            fheon_ct *out = outs[i];
            for (u32 gg = 0; gg < gn; gg++) {
                const fheon_ct *term = ly->s[g0 + gg] != 0 ? w[GC + gg] : w[gg];
                if (g0 + gg == 0) {
                    if ((rc = fheon_drop_level(ctx, term, term->level, out))) return rc;
                } else if ((rc = fheon_add(ctx, out, term, out))) {
                    return rc;
                }
            }
        }
    }
    for (u32 i = 0; i < n; i++)
        if (ly->bias && (rc = fheon_add_plain(ctx, outs[i], ly->bias, outs[i]))) return rc;
    return FHEON_OK;
}

// n inputs at once: the slot sums of all neurons of all inputs rotate together
int fc_apply(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins, u32 n, fheon_ct *const *outs)
{
    const u32 m = (u32)ly->fw.size();
    const size_t nm = (size_t)n * m;
    int rc;
    if ((rc = ensure_cts(ctx, ly->work, 2 * nm, ins[0]->level, ins[0]->scale))) return rc;
    fheon_ct *const *t = ly->work.data(), *const *u = ly->work.data() + nm;
    for (u32 i = 0; i < n; i++)
        for (u32 k = 0; k < m; k++) {
            fheon_ct *x = t[(size_t)i * m + k];
            if ((rc = fheon_mul_plain(ctx, ins[i], ly->fw[k], x))) return rc;
            if ((rc = fheon_rescale(ctx, x, x))) return rc;
        }
    std::vector<fheon_rot_item> items(nm);
    for (u32 st = 1; st < ly->nslots; st <<= 1) {
        for (size_t x = 0; x < nm; x++) items[x] = fheon_rot_item{t[x], u[x], (int32_t)st};
        if ((rc = rotate_many(ctx, items.data(), (u32)nm, false, ly->collect))) return rc;
        for (size_t x = 0; x < nm; x++)
            if ((rc = fheon_add(ctx, t[x], u[x], t[x]))) return rc;
    }
    std::vector<const fheon_pt *> es(ly->fe.begin(), ly->fe.end());
    for (u32 i = 0; i < n; i++) {
        std::vector<const fheon_ct *> ts(t + (size_t)i * m, t + (size_t)(i + 1) * m);
        if ((rc = fheon_mac_plain(ctx, ts.data(), es.data(), m, outs[i]))) return rc;
        if ((rc = fheon_rescale(ctx, outs[i], outs[i]))) return rc;
        if (ly->bias && (rc = fheon_add_plain(ctx, outs[i], ly->bias, outs[i]))) return rc;
    }
    return FHEON_OK;
}

// the largest power of two (at most n) dividing every offset
u32 common_stride(u32 n, const std::set<u32> &offs)
{
    u32 stride = n;
    for (u32 o : offs)
        while (stride > 1 && o % stride) stride /= 2;
    return stride;
}

// where every (c, i, j) of map a moves to reach its slot in map b: offset o
// = (src - dst) mod n, the destination slots of each offset
bool repack_offsets(u32 n, const fheon_map &a, const fheon_map &b, std::map<u32, std::vector<u32>> &dst_of)
{
    for (u32 c = 0; c < a.C; c++)
        for (u32 i = 0; i < a.H; i++)
            for (u32 j = 0; j < a.W; j++) {
                const u32 src = map_slot(a, c, i, j), dst = map_slot(b, c, i, j);
                const u32 o = (src + n - dst) % n;
                auto it = dst_of.find(o);
                if (it == dst_of.end()) {
                    if (dst_of.size() == 1024) return false;
                    it = dst_of.emplace(o, std::vector<u32>()).first;
                }
                it->second.push_back(dst);
            }
    return true;
}

int check_pt(fheon_ctx *ctx, const fheon_pt *p, u32 level, const char *what)
{
    if (p && p->level < level) return fail(ctx, FHEON_ERR_LEVEL, "%s below level %u", what, level);
    return FHEON_OK;
}

} // namespace

namespace fheon {
u32 conv_baby(u32 k, u32 C, u32 F)
{
    const u64 G = (u64)C + F - 1, taps = (u64)k * k;
    u32 best = 1;
    u64 best_cost = ~0ull;
    for (u64 B = 1; B <= G; B++) {
        const u64 cost = taps * B - 1 + 2 * ((G + B - 1) / B);
        if (cost < best_cost) {
            best_cost = cost;
            best = (u32)B;
        }
    }
    return best;
}

int repack_steps(u32 n, const fheon_map &a, const fheon_map &b, std::vector<int32_t> &steps)
{
    std::map<u32, std::vector<u32>> dst_of;
    if (!repack_offsets(n, a, b, dst_of)) return FHEON_ERR_ARG;
    std::set<u32> offs;
    for (auto &kv : dst_of) offs.insert(kv.first);
    const u32 stride = common_stride(n, offs);
    int64_t bs = 0;
    std::set<int64_t> ts, cs;
    bsgs_split(bsgs_offsets(offs, n, stride), (int64_t)(n / stride), 0, bs, ts, cs);
    std::set<int32_t> st;
    for (int64_t t : ts)
        if (t) st.insert((int32_t)(t * stride));
    for (int64_t c : cs)
        if (c) st.insert((int32_t)(c * bs * (int64_t)stride));
    steps.assign(st.begin(), st.end());
    return FHEON_OK;
}
} // namespace fheon

extern "C" {

int fheon_linear_prepare_plain(fheon_ctx *ctx, uint32_t nf, const int32_t *fold, uint32_t nt, const int32_t *r,
                               uint32_t ng, const int32_t *s, const fheon_pt *const *pts, const fheon_pt *bias,
                               uint32_t level, fheon_layer **out)
{
    if (!ctx || !out || !nt || !ng || !r || !s || !pts || (nf && !fold) || level < 2 || level > ctx->L)
        return FHEON_ERR_ARG;
    std::set<int32_t> seen;
    for (u32 t = 0; t < nt; t++)
        if (!seen.insert(r[t]).second) return fail(ctx, FHEON_ERR_ARG, "linear: tap step %d repeated", r[t]);
    int rc;
    for (u32 g = 0; g < ng; g++) {
        bool any = false;
        for (u32 t = 0; t < nt; t++) {
            const fheon_pt *p = pts[(size_t)g * nt + t];
            any = any || p;
            if ((rc = check_pt(ctx, p, level, "linear: plaintext"))) return rc;
        }
        if (!any) return fail(ctx, FHEON_ERR_ARG, "linear: group %u has no plaintext", g);
    }
    if ((rc = check_pt(ctx, bias, level - 1, "linear: bias"))) return rc;
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_LINEAR;
    ly->level = level;
    ly->r.assign(r, r + nt);
    ly->s.assign(s, s + ng);
    if (nf) ly->fold.assign(fold, fold + nf);
    for (size_t i = 0; i < (size_t)nt * ng; i++) ly->pts.push_back(const_cast<fheon_pt *>(pts[i]));
    ly->bias = const_cast<fheon_pt *>(bias);
    *out = ly.release();
    return FHEON_OK;
}

int fheon_fc_prepare_plain(fheon_ctx *ctx, uint32_t m, const fheon_pt *const *W, const fheon_pt *const *E,
                           const fheon_pt *bias, uint32_t level, fheon_layer **out)
{
    if (!ctx || !out || !m || !W || !E || level < 3 || level > ctx->L) return FHEON_ERR_ARG;
    int rc;
    for (u32 k = 0; k < m; k++) {
        if (!W[k] || !E[k]) return fail(ctx, FHEON_ERR_ARG, "fc: neuron %u without plaintexts", k);
        if ((rc = check_pt(ctx, W[k], level, "fc: weights"))) return rc;
        if ((rc = check_pt(ctx, E[k], level - 1, "fc: placement"))) return rc;
    }
    if ((rc = check_pt(ctx, bias, level - 2, "fc: bias"))) return rc;
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_FC;
    ly->level = level;
    ly->nslots = ctx->N / 2;
    for (u32 k = 0; k < m; k++) {
        ly->fw.push_back(const_cast<fheon_pt *>(W[k]));
        ly->fe.push_back(const_cast<fheon_pt *>(E[k]));
    }
    ly->bias = const_cast<fheon_pt *>(bias);
    ly->out_map = fheon_map{1, 1, m, m, 1, m};
    *out = ly.release();
    return FHEON_OK;
}

int fheon_conv_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t F, uint32_t k, uint32_t stride, uint32_t pad,
                       const double *K, const double *bias, uint32_t level, double in_scale, fheon_layer **out)
{
    if (!ctx || !in || !out || !K || !F || !k || !stride || level < 2 || level > ctx->L) return FHEON_ERR_ARG;
    const fheon_map im = *in;
    if (!map_ok(ctx, im) || im.H + 2 * pad < k || im.W + 2 * pad < k)
        return fail(ctx, FHEON_ERR_ARG, "conv: map does not fit the slots or the kernel");
    const u32 C = im.C, Ho = (im.H + 2 * pad - k) / stride + 1, Wo = (im.W + 2 * pad - k) / stride + 1, n = ctx->N / 2;
    // outputs at input-grid positions (stride*i, stride*j): the striding is in the weights
    const fheon_map om{F, Ho, Wo, im.grid, im.dil * stride, im.block};
    if (!map_ok(ctx, om)) return fail(ctx, FHEON_ERR_ARG, "conv: output map does not fit the slots");
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_LINEAR;
    ly->level = level;
    ly->in_map = im;
    ly->out_map = om;
    // block shift delta = a + B*b: baby a in [0, B) taken by the hoisted tap
    // rotations r_t - a*block, giant b by the group's rotation -B*b*block
    const u32 B = fheon::conv_baby(k, C, F);
    std::vector<int32_t> tap;
    for (u32 x = 0; x < k; x++)
        for (u32 y = 0; y < k; y++)
            tap.push_back((int32_t)im.dil * (((int32_t)x - (int32_t)pad) * (int32_t)im.grid + ((int32_t)y - (int32_t)pad)));
    // the layer's tap steps r - a*block, each once: on a map whose taps span
    // more than a block, two (a, tap) pairs can share a step, and their vectors
    // are summed (in (a, tap) order) into that step's plaintext
    std::vector<u32> tix; // (a, tap) -> index into ly->r
    for (u32 a = 0; a < B; a++)
        for (int32_t r : tap) {
            const int32_t st = r - (int32_t)(a * im.block);
            auto it = std::find(ly->r.begin(), ly->r.end(), st);
            tix.push_back((u32)(it - ly->r.begin()));
            if (it == ly->r.end()) ly->r.push_back(st);
        }
    const u32 nt = (u32)ly->r.size();
    const double ps = (double)ctx->mod[level - 1];
    std::vector<double> v(n);
    // adds the weights of block shift delta, tap (x, y), in the input channels'
    // blocks, moved by a*block (Rot_{-a*block}), into acc; true when any is nonzero
    auto add_group_vec = [&](int delta, u32 x, u32 y, u32 a, std::vector<double> &acc) {
        bool any = false;
        for (u32 c = 0; c < C; c++) {
            const int f = (int)c + delta;
            if (f < 0 || f >= (int)F) continue;
            const double w = K[(((size_t)f * C + c) * k + x) * k + y];
            if (w == 0.0) continue;
            for (u32 i = 0; i < Ho; i++)
                for (u32 j = 0; j < Wo; j++) {
                    const int si = (int)(stride * i + x) - (int)pad, sj = (int)(stride * j + y) - (int)pad;
                    if (si >= 0 && si < (int)im.H && sj >= 0 && sj < (int)im.W) {
                        double &d = acc[(map_slot(om, c, i, j) + (size_t)a * im.block) % n];
                        d = d + w;
                        any = true;
                    }
                }
        }
        return any;
    };
    const int dmin = -(int)(C - 1), dmax = (int)F - 1;
    auto fdiv = [](int x, int d) { return x >= 0 ? x / d : -((-x + d - 1) / d); };
    std::vector<std::vector<double>> acc(nt, std::vector<double>(n));
    std::vector<char> used(nt);
    int rc;
    for (int b = fdiv(dmin, (int)B); b <= fdiv(dmax, (int)B); b++) {
        for (auto &w : acc) std::fill(w.begin(), w.end(), 0.0);
        std::fill(used.begin(), used.end(), 0);
        for (u32 a = 0; a < B; a++) {
            const int delta = (int)a + (int)B * b;
            if (delta < dmin || delta > dmax) continue;
            for (u32 x = 0; x < k; x++)
                for (u32 y = 0; y < k; y++) {
                    const u32 t = tix[(size_t)a * k * k + x * k + y];
                    if (add_group_vec(delta, x, y, a, acc[t])) used[t] = 1;
                }
        }
        std::vector<fheon_pt *> gp(nt, nullptr);
        bool any = false;
        for (u32 t = 0; t < nt; t++) {
            if (!used[t]) continue;
            if ((rc = own_plain(ctx, ly.get(), acc[t], level, ps, &gp[t]))) return rc;
            any = any || gp[t];
        }
        if (!any) continue;
        ly->s.push_back(-b * (int32_t)B * (int32_t)im.block);
        ly->pts.insert(ly->pts.end(), gp.begin(), gp.end());
    }
    if (bias) {
        std::fill(v.begin(), v.end(), 0.0);
        for (u32 f = 0; f < F; f++)
            for (u32 i = 0; i < Ho; i++)
                for (u32 j = 0; j < Wo; j++) v[map_slot(om, f, i, j)] = bias[f];
        if ((rc = own_plain(ctx, ly.get(), v, level - 1, in_scale, &ly->bias))) return rc;
    }
    *out = ly.release();
    return FHEON_OK;
}

int fheon_avgpool_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t k, uint32_t stride, uint32_t level,
                          fheon_layer **out)
{
    if (!ctx || !in || !out || !k || !stride || level < 2 || level > ctx->L) return FHEON_ERR_ARG;
    const fheon_map im = *in;
    if (!map_ok(ctx, im) || im.H < k || im.W < k) return fail(ctx, FHEON_ERR_ARG, "avgpool: map does not fit");
    const u32 Ho = (im.H - k) / stride + 1, Wo = (im.W - k) / stride + 1, n = ctx->N / 2;
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_LINEAR;
    ly->level = level;
    ly->in_map = im;
    ly->out_map = fheon_map{im.C, Ho, Wo, im.grid, im.dil * stride, im.block};
    std::vector<double> v(n, 0.0);
    for (u32 c = 0; c < im.C; c++)
        for (u32 i = 0; i < Ho; i++)
            for (u32 j = 0; j < Wo; j++) v[map_slot(ly->out_map, c, i, j)] = 1.0 / ((double)k * k);
    fheon_pt *mask = nullptr;
    int rc = own_plain(ctx, ly.get(), v, level, (double)ctx->mod[level - 1], &mask);
    if (rc) return rc;
    for (u32 x = 0; x < k; x++)
        for (u32 y = 0; y < k; y++) {
            ly->r.push_back((int32_t)(im.dil * (x * im.grid + y)));
            ly->pts.push_back(mask);
        }
    ly->s.push_back(0);
    *out = ly.release();
    return FHEON_OK;
}

int fheon_fc_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t m, const double *W, const double *bias,
                     uint32_t level, double in_scale, fheon_layer **out)
{
    if (!ctx || !in || !out || !W || !m || m > ctx->N / 2 || level < 2 || level > ctx->L) return FHEON_ERR_ARG;
    const fheon_map im = *in;
    if (!map_ok(ctx, im)) return fail(ctx, FHEON_ERR_ARG, "fc: map does not fit");
    const u32 n = ctx->N / 2, C = im.C, nin = C * im.H * im.W;
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_LINEAR;
    ly->level = level;
    ly->in_map = im;
    ly->out_map = fheon_map{1, 1, m, m, 1, m};
    // fold the channels into block 0 when they interleave on the dilation grid
    std::vector<int64_t> off(C);
    bool fold = im.dil >= 2 && C <= im.dil * im.dil && im.dil * im.W <= im.grid;
    for (u32 c = 0; c < C && fold; c++) off[c] = (int64_t)(c % im.dil) + (int64_t)im.grid * (c / im.dil);
    if (fold && off[C - 1] + (int64_t)im.dil * ((int64_t)(im.H - 1) * im.grid + (im.W - 1)) >= (int64_t)im.block)
        fold = false;
    for (u32 c = 0; c < C; c++) {
        if (!fold) off[c] = (int64_t)c * im.block;
        else ly->fold.push_back((int32_t)((int64_t)c * im.block - off[c]));
    }
    std::vector<int64_t> slot(nin);
    for (u32 c = 0, t = 0; c < C; c++)
        for (u32 i = 0; i < im.H; i++)
            for (u32 j = 0; j < im.W; j++) slot[t++] = off[c] + (int64_t)im.dil * ((int64_t)i * im.grid + j);
    int64_t smin = slot[0], smax = slot[0];
    for (int64_t v : slot) smin = std::min(smin, v), smax = std::max(smax, v);
    // y[k] = sum_d diag_d[k] x'[k + d], d = e_g + a (baby steps a < b, giant steps e_g)
    const int64_t dmin = smin - (int64_t)(m - 1), span = smax - dmin + 1;
    const int64_t b = (int64_t)std::ceil(std::sqrt((double)span)), ng = (span + b - 1) / b;
    for (int64_t a = 0; a < b; a++) ly->r.push_back((int32_t)a);
    // inputs t by slot, to find the input at slot k + d
    std::vector<int32_t> at((size_t)(smax - smin + 1), -1);
    for (u32 t = 0; t < nin; t++) at[(size_t)(slot[t] - smin)] = (int32_t)t;
    const double ps = (double)ctx->mod[level - 1];
    std::vector<double> v(n);
    int rc;
    for (int64_t g = 0; g < ng; g++) {
        const int64_t e = dmin + g * b;
        std::vector<fheon_pt *> gp;
        bool any = false;
        for (int64_t a = 0; a < b; a++) {
            const int64_t d = e + a;
            std::fill(v.begin(), v.end(), 0.0);
            for (u32 k = 0; k < m; k++) {
                const int64_t sl = (int64_t)k + d;
                if (sl < smin || sl > smax) continue;
                const int32_t t = at[(size_t)(sl - smin)];
                if (t < 0) continue;
                // the plaintext is Rot_{-e}(diag_d): diag_d[k] lands at slot k + e
                v[(size_t)((((int64_t)k + e) % (int64_t)n + (int64_t)n) % (int64_t)n)] = W[(size_t)k * nin + t];
            }
            fheon_pt *p = nullptr;
            if ((rc = own_plain(ctx, ly.get(), v, level, ps, &p))) return rc;
            gp.push_back(p);
            any = any || p;
        }
        if (!any) continue;
        ly->s.push_back((int32_t)e);
        ly->pts.insert(ly->pts.end(), gp.begin(), gp.end());
    }
    if (bias) {
        std::fill(v.begin(), v.end(), 0.0);
        for (u32 k = 0; k < m; k++) v[k] = bias[k];
        if ((rc = own_plain(ctx, ly.get(), v, level - 1, in_scale, &ly->bias))) return rc;
    }
    *out = ly.release();
    return FHEON_OK;
}

int fheon_repack_prepare(fheon_ctx *ctx, const fheon_map *in, const fheon_map *out, uint32_t level,
                         fheon_layer **layer)
{
    if (!ctx || !in || !out || !layer || level < 2 || level > ctx->L) return FHEON_ERR_ARG;
    const fheon_map a = *in, b = *out;
    if (!map_ok(ctx, a) || !map_ok(ctx, b) || a.C != b.C || a.H != b.H || a.W != b.W)
        return fail(ctx, FHEON_ERR_ARG, "repack: maps of the same (C, H, W) that fit the slots");
    const u32 n = ctx->N / 2;
    // every (c, i, j) moves from its slot in `in` to its slot in `out`:
    // out = sum_o m_o Rot_o(in), m_o one at each destination o slots before its source
    std::map<u32, std::vector<u32>> dst_of;
    if (!repack_offsets(n, a, b, dst_of))
        return fail(ctx, FHEON_ERR_ARG, "repack: more than 1024 distinct shifts; split it");
    Diags D;
    std::set<u32> offs;
    for (auto &kv : dst_of) {
        std::vector<cd> &d = D.emplace(kv.first, std::vector<cd>(n, cd(0.0))).first->second;
        for (u32 dst : kv.second) d[dst] = cd(1.0);
        offs.insert(kv.first);
    }
    int rc = diag_layer(ctx, D, common_stride(n, offs), cd(1.0), 0, level, (double)ctx->mod[level - 1], layer);
    if (rc) return rc;
    (*layer)->in_map = a;
    (*layer)->out_map = b;
    return FHEON_OK;
}

int fheon_global_avgpool_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t level, fheon_layer **out)
{
    if (!ctx || !in || in->H != in->W) return FHEON_ERR_ARG;
    return fheon_avgpool_prepare(ctx, in, in->H, in->H, level, out);
}

// the FC layer as the paper states it: one product per neuron, the sum of its
// slots by rotate-and-add, a one-hot placement (log2(N/2) keys)
static int fc_slot_sum_prepare(fheon_ctx *ctx, const fheon_map *in, uint32_t m, const double *W, const double *bias,
                               uint32_t level, double in_scale, fheon_layer **out)
{
    if (level < 3) return fail(ctx, FHEON_ERR_LEVEL, "fc: the slot-sum form needs level >= 3");
    const fheon_map im = *in;
    const u32 n = ctx->N / 2, nin = im.C * im.H * im.W;
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_FC;
    ly->level = level;
    ly->nslots = n;
    ly->in_map = im;
    ly->out_map = fheon_map{1, 1, m, m, 1, m};
    std::vector<u32> slots;
    for (u32 c = 0; c < im.C; c++)
        for (u32 i = 0; i < im.H; i++)
            for (u32 j = 0; j < im.W; j++) slots.push_back(map_slot(im, c, i, j));
    std::vector<double> v(n);
    int rc;
    for (u32 k = 0; k < m; k++) {
        std::fill(v.begin(), v.end(), 0.0);
        for (u32 t = 0; t < nin; t++) v[slots[t]] = W[(size_t)k * nin + t];
        fheon_pt *w = nullptr, *e = nullptr;
        if ((rc = own_plain(ctx, ly.get(), v, level, (double)ctx->mod[level - 1], &w))) return rc;
        if (!w) return fail(ctx, FHEON_ERR_ARG, "fc: neuron %u has all-zero weights", k);
        std::fill(v.begin(), v.end(), 0.0);
        v[k] = 1.0;
        if ((rc = own_plain(ctx, ly.get(), v, level - 1, (double)ctx->mod[level - 2], &e))) return rc;
        ly->fw.push_back(w);
        ly->fe.push_back(e);
    }
    if (bias) {
        std::fill(v.begin(), v.end(), 0.0);
        for (u32 k = 0; k < m; k++) v[k] = bias[k];
        if ((rc = own_plain(ctx, ly.get(), v, level - 2, in_scale, &ly->bias))) return rc;
    }
    *out = ly.release();
    return FHEON_OK;
}

int fheon_fc(fheon_ctx *ctx, const fheon_ct *ct, const fheon_map *in, uint32_t m, const double *W, const double *bias,
             uint32_t max_keys, fheon_ct *out)
{
    if (!ctx || !ct || !in || !out) return FHEON_ERR_ARG;
    fheon_layer *ly = nullptr;
    int rc = fheon_fc_prepare(ctx, in, m, W, bias, ct->level, ct->scale, &ly);
    if (rc) return rc;
    uint32_t nk = 0;
    fheon_layer_rotation_steps(ly, nullptr, &nk);
    if (max_keys && nk > max_keys) {
        // the paper's form needs log2(N/2) keys
        fheon_layer_destroy(ly);
        ly = nullptr;
        u32 lg = 0;
        while ((1u << lg) < ctx->N / 2) lg++;
        if (lg > max_keys) return fail(ctx, FHEON_ERR_ARG, "fc: needs at least %u rotation keys", lg);
        if ((rc = fc_slot_sum_prepare(ctx, in, m, W, bias, ct->level, ct->scale, &ly))) return rc;
    }
    rc = fheon_layer_apply(ctx, ly, ct, out);
    fheon_layer_destroy(ly);
    return rc;
}

int fheon_avgpool(fheon_ctx *ctx, const fheon_ct *ct, const fheon_map *in, uint32_t k, uint32_t stride, fheon_ct *out)
{
    if (!ctx || !ct) return FHEON_ERR_ARG;
    fheon_layer *ly = nullptr;
    int rc = fheon_avgpool_prepare(ctx, in, k, stride, ct->level, &ly);
    if (rc) return rc;
    rc = fheon_layer_apply(ctx, ly, ct, out);
    fheon_layer_destroy(ly);
    return rc;
}

int fheon_global_avgpool(fheon_ctx *ctx, const fheon_ct *ct, const fheon_map *in, fheon_ct *out)
{
    if (!ctx || !ct) return FHEON_ERR_ARG;
    fheon_layer *ly = nullptr;
    int rc = fheon_global_avgpool_prepare(ctx, in, ct->level, &ly);
    if (rc) return rc;
    rc = fheon_layer_apply(ctx, ly, ct, out);
    fheon_layer_destroy(ly);
    return rc;
}

int fheon_layer_apply(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !ly || !in || !out) return FHEON_ERR_ARG;
    return fheon_layer_apply_batch(ctx, ly, &in, 1, &out);
}

int fheon_layer_apply_batch(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins, uint32_t n,
                            fheon_ct *const *outs)
{
    if (!ctx || !ly || (n && (!ins || !outs))) return FHEON_ERR_ARG;
    if (n == 0) return FHEON_OK;
    std::set<const void *> in_set;
    for (u32 i = 0; i < n; i++) {
        if (!ins[i] || !outs[i]) return fail(ctx, FHEON_ERR_ARG, "layer batch: null ciphertext %u", i);
        in_set.insert(ins[i]);
    }
    std::set<const void *> out_set;
    for (u32 i = 0; i < n; i++) {
        if (in_set.count(outs[i])) return fail(ctx, FHEON_ERR_ARG, "layer output %u aliases an input", i);
        if (!out_set.insert(outs[i]).second) return fail(ctx, FHEON_ERR_ARG, "layer output %u repeated", i);
    }
    static const char *const kind_name[] = {"layer_conv", "layer_relu", "layer_linear", "layer_fc", "layer_bootstrap"};
    Range range(ly->kind <= LAYER_BOOT ? kind_name[ly->kind] : "layer");
    int rc;
    switch (ly->kind) {
    case LAYER_CONV:
        for (u32 i = 0; i < n; i++)
            if ((rc = fheon_conv2d_apply(ctx, ly, ins[i], outs[i]))) return rc;
        return FHEON_OK;
    case LAYER_RELU:
        return relu_apply_batch(ctx, ly, ins, n, outs);
    case LAYER_BOOT:
        return n == 1 ? boot_apply(ctx, ly, ins[0], outs[0]) : boot_apply_many(ctx, ly, ins, n, outs);
    default: break;
    }
    for (u32 i = 0; i < n; i++)
        if (ins[i]->level != ly->level)
            return fail(ctx, FHEON_ERR_LEVEL, "layer expects level %u, got %u", ly->level, ins[i]->level);
    return ly->kind == LAYER_LINEAR ? linear_apply(ctx, ly, ins, n, outs) : fc_apply(ctx, ly, ins, n, outs);
}

int fheon_layer_rotation_steps(const fheon_layer *ly, int32_t *out, uint32_t *n)
{
    if (!ly || !n) return FHEON_ERR_ARG;
    std::set<int32_t> st;
    if (ly->kind == LAYER_LINEAR) {
        for (int32_t x : ly->fold)
            if (x) st.insert(x);
        for (int32_t x : ly->r)
            if (x) st.insert(x);
        for (int32_t x : ly->s)
            if (x) st.insert(x);
    } else if (ly->kind == LAYER_FC) {
        for (u32 x = 1; x < ly->nslots; x <<= 1) st.insert((int32_t)x);
    } else if (ly->kind == LAYER_BOOT) {
        // sparse: the copies' rotations n_s, 2 n_s, ... (repetition and trace)
        if (ly->boot_ns)
            for (u32 x = ly->boot_ns; x < ly->nslots; x <<= 1) st.insert((int32_t)x);
        for (const fheon_layer *sub : ly->subs) {
            for (int32_t x : sub->r)
                if (x) st.insert(x);
            for (int32_t x : sub->s)
                if (x) st.insert(x);
        }
    } else if (ly->kind == LAYER_CONV) {
        const int p = (int)(ly->k - 1) / 2;
        for (int di = -p; di <= p; di++)
            for (int dj = -p; dj <= p; dj++)
                if (di || dj) st.insert(di * (int)ly->W + dj);
        if (ly->in_ch > 1) st.insert((int32_t)(ly->H * ly->W));
    }
    const uint32_t cap = *n;
    *n = (uint32_t)st.size();
    if (out && cap < st.size()) return FHEON_ERR_ARG;
    if (out) {
        u32 i = 0;
        for (int32_t x : st) out[i++] = x;
    }
    return FHEON_OK;
}

int fheon_layer_out_map(const fheon_layer *ly, fheon_map *out)
{
    if (!ly || !out || (ly->kind != LAYER_LINEAR && ly->kind != LAYER_FC)) return FHEON_ERR_ARG;
    *out = ly->out_map;
    return FHEON_OK;
}

} // extern "C"
