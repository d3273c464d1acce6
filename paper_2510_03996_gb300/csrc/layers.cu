// layers.cu -- FHEON's special secure convolution (paper Sec. 5.3, Alg. 1-3),
// generalised from 3x3 to any odd k with "same" padding and stride 1, as host
// orchestration of the device operations.
//
// Input packing (paper Sec. 5.1, flattening): channel c, row h, column w at
// slot c*H*W + h*W + w.  For tap (di, dj) in [-p, p]^2, p = (k-1)/2, the
// rotated ciphertext Rot_{di*W+dj}(x) holds x[h+di][w+dj] at slot (h, w); the
// tap plaintext is the kernel value times the boundary mask of Alg. 2/3
// (1 where (h+di, w+dj) lies inside the input), per channel block.  The
// k^2 - 1 tap rotations of the input are hoisted (one raising of c1 shared by
// all of them: the "fast rotations" of Sec. 3.2); the k^2 products are formed
// and summed in one pass and rescaled once (the taps are encoded at scale
// q_{level-1}, so the scale returns to the input's).  With C > 1 input
// channels the channel blocks are summed by C-1 chained rotations by H*W
// (the single W^2 key of Sec. 5.3) and masked to block 0, which costs one
// more level.  The bias is added last.
#include <algorithm>
#include <cmath>
#include <memory>
#include <set>
#include <vector>

#include "layer.h"

using namespace fheon;

namespace {
struct CtGuard {
    fheon_ct *p = nullptr;
    ~CtGuard() { fheon_ct_destroy(p); }
};

bool conv2d_is_special(u32 in_ch, u32 out_ch, u32 k, u32 stride, u32 pad)
{
    return in_ch == 1 && out_ch == 1 && k % 2 == 1 && stride == 1 && pad == (k - 1) / 2;
}

bool same_map(const fheon_map &a, const fheon_map &b)
{
    return a.C == b.C && a.H == b.H && a.W == b.W && a.grid == b.grid && a.dil == b.dil && a.block == b.block;
}

// the output map of the rotation-sum conv on the compact (C, H, W) input (its
// outputs at the stride-aligned slots of the input grid) and the compact
// output map (F, Ho, Wo) the one-shot call returns
void conv2d_maps(u32 C, u32 F, u32 k, u32 stride, u32 pad, u32 H, u32 W, fheon_map &om, fheon_map &cm)
{
    const u32 Ho = (H + 2 * pad - k) / stride + 1, Wo = (W + 2 * pad - k) / stride + 1;
    (void)C;
    om = fheon_map{F, Ho, Wo, W, stride, H * W};
    cm = fheon_map{F, Ho, Wo, Wo, 1, Ho * Wo};
}

int make_mask(fheon_ctx *ctx, fheon_layer *ly)
{
    if (ly->in_ch <= 1) return FHEON_OK;
    if (ly->level < 3) return fail(ctx, FHEON_ERR_LEVEL, "multi-channel conv needs level >= 3");
    const u32 n = ctx->N / 2, hw = ly->H * ly->W;
    std::vector<double> v(n, 0.0);
    for (u32 s = 0; s < hw; s++) v[s] = 1.0;
    const u32 lv = ly->level - 1;
    return fheon_encode_plain(ctx, v.data(), nullptr, n, lv, (double)ctx->mod[lv - 1], &ly->mask);
}
} // namespace

extern "C" {

int fheon_conv2d_rotation_steps(uint32_t N, uint32_t in_ch, uint32_t out_ch, uint32_t k, uint32_t stride,
                                uint32_t pad, uint32_t in_h, uint32_t in_w, int32_t *out, uint32_t *n)
{
    if (!n || in_ch == 0 || out_ch == 0 || k == 0 || stride == 0 || in_h == 0 || in_w == 0 || N < 2 || (N & (N - 1)))
        return FHEON_ERR_ARG;
    if (in_h + 2 * pad < k || in_w + 2 * pad < k) return FHEON_ERR_ARG;
    std::set<int32_t> s;
    if (conv2d_is_special(in_ch, out_ch, k, stride, pad)) {
        const int p = (int)(k - 1) / 2;
        for (int di = -p; di <= p; di++)
            for (int dj = -p; dj <= p; dj++)
                if (di || dj) s.insert(di * (int)in_w + dj);
    } else {
        // the rotation-sum conv on the compact map (taps, block shifts), then the
        // repack of its output to the compact (F, Ho, Wo) layout when needed
        const u32 nsl = N / 2, block = in_h * in_w;
        if ((u64)std::max(in_ch, out_ch) * block > nsl) return FHEON_ERR_ARG;
        // the plan's hoisted taps r - a*block (a < B) and giant steps -B*b*block
        const u32 B = conv_baby(k, in_ch, out_ch);
        for (u32 a = 0; a < B; a++)
            for (u32 x = 0; x < k; x++)
                for (u32 y = 0; y < k; y++) {
                    const int32_t r = ((int32_t)x - (int32_t)pad) * (int32_t)in_w + ((int32_t)y - (int32_t)pad) -
                                      (int32_t)(a * block);
                    if (r) s.insert(r);
                }
        auto fdiv = [](int x, int d) { return x >= 0 ? x / d : -((-x + d - 1) / d); };
        for (int b = fdiv(-(int)(in_ch - 1), (int)B); b <= fdiv((int)out_ch - 1, (int)B); b++)
            if (b) s.insert(-b * (int32_t)B * (int32_t)block);
        fheon_map om, cm;
        conv2d_maps(in_ch, out_ch, k, stride, pad, in_h, in_w, om, cm);
        if (!same_map(om, cm)) {
            std::vector<int32_t> rs;
            if (repack_steps(nsl, om, cm, rs)) return FHEON_ERR_ARG;
            s.insert(rs.begin(), rs.end());
        }
    }
    const u32 cap = *n;
    *n = (u32)s.size();
    if (out && cap < s.size()) return FHEON_ERR_ARG;
    if (out) {
        u32 i = 0;
        for (int32_t x : s) out[i++] = x;
    }
    return FHEON_OK;
}

int fheon_conv2d_prepare(fheon_ctx *ctx, uint32_t in_ch, uint32_t k, uint32_t stride, uint32_t pad, uint32_t in_h,
                         uint32_t in_w, const double *w, const double *bias, uint32_t level, double in_scale,
                         fheon_layer **out)
{
    if (!ctx || !w || !out || in_ch == 0 || k == 0 || in_h == 0 || in_w == 0 || level < 2 || level > ctx->L)
        return FHEON_ERR_ARG;
    if (k % 2 == 0 || stride != 1 || pad != (k - 1) / 2)
        return fail(ctx, FHEON_ERR_UNIMPLEMENTED, "only the special conv (odd k, stride 1, pad (k-1)/2) is built");
    const u32 n = ctx->N / 2, hw = in_h * in_w;
    if ((u64)in_ch * hw > n) return fail(ctx, FHEON_ERR_ARG, "input does not fit in %u slots", n);
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->in_ch = in_ch;
    ly->k = k;
    ly->H = in_h;
    ly->W = in_w;
    ly->level = level;
    const int p = (int)(k - 1) / 2;
    const double tap_scale = (double)ctx->mod[level - 1];
    std::vector<double> v(n);
    for (int di = -p; di <= p; di++)
        for (int dj = -p; dj <= p; dj++) {
            std::fill(v.begin(), v.end(), 0.0);
            for (u32 c = 0; c < in_ch; c++) {
                const double kv = w[((size_t)c * k + (di + p)) * k + (dj + p)];
                for (u32 h = 0; h < in_h; h++)
                    for (u32 x = 0; x < in_w; x++) {
                        const int hh = (int)h + di, xx = (int)x + dj;
                        if (hh >= 0 && hh < (int)in_h && xx >= 0 && xx < (int)in_w) v[c * hw + h * in_w + x] = kv;
                    }
            }
            fheon_pt *pt = nullptr;
            int rc = fheon_encode_plain(ctx, v.data(), nullptr, n, level, tap_scale, &pt);
            if (rc) return rc;
            ly->taps.push_back(pt);
            ly->owned.push_back(true);
        }
    int rc = make_mask(ctx, ly.get());
    if (rc) return rc;
    if (bias) {
        std::fill(v.begin(), v.end(), 0.0);
        for (u32 s = 0; s < hw; s++) v[s] = bias[0];
        const u32 out_level = level - (in_ch > 1 ? 2 : 1);
        rc = fheon_encode_plain(ctx, v.data(), nullptr, n, out_level, in_scale, &ly->bias);
        if (rc) return rc;
        ly->own_bias = true;
    }
    *out = ly.release();
    return FHEON_OK;
}

int fheon_conv2d_prepare_plain(fheon_ctx *ctx, uint32_t in_ch, uint32_t k, uint32_t in_h, uint32_t in_w,
                               uint32_t level, const fheon_pt *const *taps, const fheon_pt *bias, fheon_layer **out)
{
    if (!ctx || !taps || !out || k % 2 == 0 || in_ch == 0 || level < 2 || level > ctx->L) return FHEON_ERR_ARG;
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->in_ch = in_ch;
    ly->k = k;
    ly->H = in_h;
    ly->W = in_w;
    ly->level = level;
    for (u32 t = 0; t < k * k; t++) {
        if (!taps[t] || taps[t]->level < level) return fail(ctx, FHEON_ERR_LEVEL, "tap %u missing or below level", t);
        ly->taps.push_back(const_cast<fheon_pt *>(taps[t]));
        ly->owned.push_back(false);
    }
    ly->bias = const_cast<fheon_pt *>(bias);
    int rc = make_mask(ctx, ly.get());
    if (rc) return rc;
    *out = ly.release();
    return FHEON_OK;
}

int fheon_conv2d_apply(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !ly || !in || !out || ly->kind != LAYER_CONV) return FHEON_ERR_ARG;
    if (in->level != ly->level) return fail(ctx, FHEON_ERR_LEVEL, "conv expects level %u, got %u", ly->level, in->level);
    if (out == in) return fail(ctx, FHEON_ERR_ARG, "conv output must not alias its input");
    const int p = (int)(ly->k - 1) / 2;
    const u32 kk = ly->k * ly->k;
    int rc;
    for (fheon_ct *&c : ly->tmp)
        if (!c && (rc = fheon_ct_create(ctx, ly->level, in->scale, &c))) return rc;
    if (ly->rot.size() != kk - 1) ly->rot.resize(kk - 1, nullptr);
    for (fheon_ct *&c : ly->rot)
        if (!c && (rc = fheon_ct_create(ctx, ly->level, in->scale, &c))) return rc;
    struct Ref {
        fheon_ct *p;
    } rot{ly->tmp[0]}, acc{ly->tmp[1]};
    // the tap rotations, hoisted; the identity tap reads the input itself
    std::vector<int32_t> steps;
    std::vector<fheon_ct *> routs;
    std::vector<const fheon_ct *> srcs;
    for (int di = -p; di <= p; di++)
        for (int dj = -p; dj <= p; dj++) {
            const int r = di * (int)ly->W + dj;
            if (r == 0) {
                srcs.push_back(in);
                continue;
            }
            if (routs.size() == ly->rot.size()) return fail(ctx, FHEON_ERR_ARG, "conv: tap rotations exceed k^2 - 1");
            steps.push_back(r);
            routs.push_back(ly->rot[routs.size()]);
            srcs.push_back(routs.back());
        }
    if ((rc = rotate_hoisted(ctx, in, steps.data(), (u32)steps.size(), routs.data(), ly->collect))) return rc;
    // the k^2 products with the tap plaintexts, summed in one pass
    if ((rc = fheon_mac_plain(ctx, srcs.data(), ly->taps.data(), kk, acc.p))) return rc;
    if (ly->in_ch > 1) {
        if ((rc = fheon_rescale(ctx, acc.p, acc.p))) return rc;
        // channel sum: acc + Rot_{HW}(acc) + Rot_{2HW}(acc) + ..., chained on one key
        if ((rc = fheon_drop_level(ctx, acc.p, acc.p->level, rot.p))) return rc;
        const int32_t hw = (int32_t)(ly->H * ly->W);
        Ref sum{ly->tmp[2]};
        if ((rc = fheon_drop_level(ctx, acc.p, acc.p->level, sum.p))) return rc;
        for (u32 c = 1; c < ly->in_ch; c++) {
            if ((rc = fheon_rotate(ctx, rot.p, hw, rot.p))) return rc;
            if ((rc = fheon_add(ctx, sum.p, rot.p, sum.p))) return rc;
        }
        if ((rc = fheon_mul_plain(ctx, sum.p, ly->mask, sum.p))) return rc;
        if ((rc = fheon_rescale(ctx, sum.p, out))) return rc;
    } else {
        if ((rc = fheon_rescale(ctx, acc.p, out))) return rc;
    }
    if (ly->bias && (rc = fheon_add_plain(ctx, out, ly->bias, out))) return rc;
    return FHEON_OK;
}

int fheon_conv2d_apply_graph(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !ly || !in || !out || ly->kind != LAYER_CONV) return FHEON_ERR_ARG;
    return fheon_layer_apply_graph(ctx, ly, in, out);
}

int fheon_layer_apply_graph(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !ly || !in || !out) return FHEON_ERR_ARG;
    if (!ctx->stream) return fail(ctx, FHEON_ERR_ARG, "graph capture needs a created stream, not the legacy default stream");
    for (auto it = ly->graphs.begin(); it != ly->graphs.end(); ++it) {
        auto &g = *it;
        if (g.in == in->c.p && g.out == out->c.p && g.ws == ctx->ws.p && g.level == in->level && g.scale == in->scale) {
            if (out->cap < g.out_level) {
                // the output buffer at this address is a newer, smaller
                // allocation than the one captured: drop the entry, capture anew
                cudaGraphExecDestroy(g.exec);
                ly->graphs.erase(it);
                break;
            }
            FHEON_CUDA(ctx, cudaGraphLaunch(g.exec, ctx->stream));
            out->level = g.out_level; // the host-side metadata the captured run set
            out->scale = g.out_scale;
            return FHEON_OK;
        }
    }
    // eager run: sizes the output, the working ciphertexts and the workspace
    int rc = fheon_layer_apply(ctx, ly, in, out);
    if (rc) return rc;
    const void *ws = ctx->ws.p;
    // capture the identical launch sequence (it allocates nothing now; the
    // rotation plans it reads are held by the graph entry)
    PlanKeep keep;
    FHEON_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ly->collect = &keep;
    rc = fheon_layer_apply(ctx, ly, in, out);
    ly->collect = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
    if (ctx->ws.p != ws) {
        cudaGraphDestroy(graph);
        return fail(ctx, FHEON_ERR_ARG, "workspace moved during capture");
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaGraphInstantiate");
    ly->graphs.push_back(fheon_layer::Graph{in->c.p, out->c.p, ctx->ws.p, in->level, in->scale, out->level,
                                            out->scale, exec, std::move(keep)});
    return FHEON_OK;
}

int fheon_conv2d(fheon_ctx *ctx, const fheon_ct *in, uint32_t in_ch, uint32_t out_ch, uint32_t k, uint32_t stride,
                 uint32_t pad, uint32_t in_h, uint32_t in_w, const double *w, const double *bias, fheon_ct *out)
{
    if (!ctx || !in || !out || !w || in_ch == 0 || out_ch == 0 || k == 0 || stride == 0 || in_h == 0 || in_w == 0)
        return FHEON_ERR_ARG;
    int rc;
    if (conv2d_is_special(in_ch, out_ch, k, stride, pad)) {
        fheon_layer *ly = nullptr;
        if ((rc = fheon_conv2d_prepare(ctx, in_ch, k, stride, pad, in_h, in_w, w, bias, in->level, in->scale, &ly)))
            return rc;
        rc = fheon_conv2d_apply(ctx, ly, in, out);
        fheon_layer_destroy(ly);
        return rc;
    }
    const fheon_map im{in_ch, in_h, in_w, in_w, 1, in_h * in_w};
    fheon_map om, cm;
    conv2d_maps(in_ch, out_ch, k, stride, pad, in_h, in_w, om, cm);
    fheon_layer *conv = nullptr;
    if ((rc = fheon_conv_prepare(ctx, &im, out_ch, k, stride, pad, w, bias, in->level, in->scale, &conv))) return rc;
    if (same_map(om, cm)) {
        rc = fheon_layer_apply(ctx, conv, in, out);
        fheon_layer_destroy(conv);
        return rc;
    }
    // the outputs sit at the stride-aligned slots of the input grid: one repack
    // makes them the compact (F, Ho, Wo) map
    CtGuard mid;
    fheon_layer *rp = nullptr;
    if ((rc = fheon_ct_create(ctx, 1, in->scale, &mid.p)) || (rc = fheon_layer_apply(ctx, conv, in, mid.p))) {
        fheon_layer_destroy(conv);
        return rc;
    }
    fheon_layer_destroy(conv);
    if (mid.p->level < 2) return fail(ctx, FHEON_ERR_LEVEL, "conv2d: the compaction needs one more level");
    if ((rc = fheon_repack_prepare(ctx, &om, &cm, mid.p->level, &rp))) return rc;
    rc = fheon_layer_apply(ctx, rp, mid.p, out);
    fheon_layer_destroy(rp);
    return rc;
}

int fheon_layer_destroy(fheon_layer *layer)
{
    delete layer;
    return FHEON_OK;
}

int fheon_layer_plan_info(const fheon_layer *ly, uint32_t *kind, uint32_t *level, uint32_t *nf, uint32_t *nt,
                          uint32_t *ng)
{
    if (!ly) return FHEON_ERR_ARG;
    u32 f = 0, t = 0, g = 0;
    switch (ly->kind) {
    case LAYER_LINEAR: f = (u32)ly->fold.size(); t = (u32)ly->r.size(); g = (u32)ly->s.size(); break;
    case LAYER_FC: g = (u32)ly->fw.size(); break;
    case LAYER_CONV: t = (u32)ly->taps.size(); g = 1; break;
    case LAYER_BOOT: t = ly->ncts; g = (u32)ly->subs.size() - ly->ncts; break;
    default: break;
    }
    if (kind) *kind = ly->kind;
    if (level) *level = ly->level;
    if (nf) *nf = f;
    if (nt) *nt = t;
    if (ng) *ng = g;
    return FHEON_OK;
}

int fheon_layer_plan(const fheon_layer *ly, int32_t *fold, int32_t *r, int32_t *s)
{
    if (!ly || ly->kind != LAYER_LINEAR) return FHEON_ERR_ARG;
    if (fold) std::copy(ly->fold.begin(), ly->fold.end(), fold);
    if (r) std::copy(ly->r.begin(), ly->r.end(), r);
    if (s) std::copy(ly->s.begin(), ly->s.end(), s);
    return FHEON_OK;
}

int fheon_layer_plain(const fheon_layer *ly, uint32_t which, uint32_t g, uint32_t t, const fheon_pt **out)
{
    if (!ly || !out) return FHEON_ERR_ARG;
    *out = nullptr;
    switch (which) {
    case FHEON_PLAIN_PRODUCT:
        if (ly->kind == LAYER_LINEAR) {
            if (g >= ly->s.size() || t >= ly->r.size()) return FHEON_ERR_ARG;
            *out = ly->pts[(size_t)g * ly->r.size() + t];
        } else if (ly->kind == LAYER_FC) {
            if (g >= ly->fw.size() || t) return FHEON_ERR_ARG;
            *out = ly->fw[g];
        } else if (ly->kind == LAYER_CONV) {
            if (g || t >= ly->taps.size()) return FHEON_ERR_ARG;
            *out = ly->taps[t];
        } else {
            return FHEON_ERR_ARG;
        }
        return FHEON_OK;
    case FHEON_PLAIN_PLACE:
        if (ly->kind != LAYER_FC || g >= ly->fe.size() || t) return FHEON_ERR_ARG;
        *out = ly->fe[g];
        return FHEON_OK;
    case FHEON_PLAIN_BIAS:
        if (g || t) return FHEON_ERR_ARG;
        *out = ly->bias;
        return FHEON_OK;
    case FHEON_PLAIN_MASK:
        if (g || t) return FHEON_ERR_ARG;
        *out = ly->mask;
        return FHEON_OK;
    case FHEON_PLAIN_MONO:
        if (ly->kind != LAYER_BOOT || g > 1 || t) return FHEON_ERR_ARG;
        *out = ly->mono[g];
        return FHEON_OK;
    case FHEON_PLAIN_BOOT_MASK:
        if (ly->kind != LAYER_BOOT || g || t) return FHEON_ERR_ARG;
        *out = ly->boot_mask;
        return FHEON_OK;
    default: return FHEON_ERR_ARG;
    }
}

int fheon_layer_sub(const fheon_layer *ly, uint32_t i, const fheon_layer **out)
{
    if (!ly || !out || ly->kind != LAYER_BOOT || i >= ly->subs.size()) return FHEON_ERR_ARG;
    *out = ly->subs[i];
    return FHEON_OK;
}

int fheon_layer_coeffs(const fheon_layer *ly, double *out, uint32_t *n)
{
    if (!ly || !n || (ly->kind != LAYER_RELU && ly->kind != LAYER_BOOT)) return FHEON_ERR_ARG;
    const u32 cap = *n;
    *n = (u32)ly->coeffs.size();
    if (out && cap < ly->coeffs.size()) return FHEON_ERR_ARG;
    if (out) std::copy(ly->coeffs.begin(), ly->coeffs.end(), out);
    return FHEON_OK;
}

} // extern "C"
