// relu.cu -- FHEON's secure ReLU (paper Sec. 5.6, Alg. 4) as host
// orchestration of the device operations: the input times a 1/beta slot mask
// (when beta > 1), then a degree-D Chebyshev series of f(z) = beta * max(0, z)
// on [-1, 1].
//
// Coefficients: Chebyshev interpolation at the D+1 nodes z_k = cos(theta_k),
// theta_k = pi (k + 1/2) / (D + 1): c_d = 2/(D+1) sum_k f(z_k) cos(d theta_k),
// c_0 halved (summed in order k = 0..D in binary64).  The paper prints the
// nodes as cos(k pi / d), which are the extrema of T_d; the interpolation nodes
// are the zeros of T_{D+1}.
//
// Evaluation (cheb_series, shared with bootstrapping's EvalMod; depth
// cheb_depth(D), 6 for degree 59, + 1 for the mask), baby steps and giant
// steps (Paterson-Stockmeyer in the Chebyshev basis):
//   babies T_1 = v, T_2h = 2 T_h^2 - 1, T_2h+1 = 2 T_h+1 T_h - T_1 up to
//   T_k (k = 2^ceil(log2(D+1)/2)), each product at the lower operand's level
//   with relinearisation, rescaled (the -T_1 of an odd one joins the product
//   before its rescale, as T_1 times K = llround(-S / s_1));
//   giants T_k, T_2k = 2 T_k^2 - 1, ..., up to m of them (D < k 2^m);
//   p = r + q T_g (g = k 2^(j-1), q_0 = c_g, q_j = 2 c_{g+j}, r_{g-j} -= c_{g+j})
//   recursively: q aimed at the scale that lands the product q T_g,
//   rescaled, on the target; a leaf (degree < k) is one integer combination
//   of the babies, rescaled once onto its target, plus c_0.
// The output has the input's scale; about 2 sqrt(D) + log2 D products.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "layer.h"

using namespace fheon;

namespace {

void relu_cheb(double beta, u32 D, std::vector<double> &c)
{
    c.assign(D + 1, 0.0);
    for (u32 d = 0; d <= D; d++) {
        double acc = 0.0;
        for (u32 k = 0; k <= D; k++) {
            const double theta = M_PI * ((double)k + 0.5) / (double)(D + 1);
            const double z = std::cos(theta);
            const double fz = z < 0.0 ? 0.0 : beta * z;
            acc += fz * std::cos((double)d * theta);
        }
        c[d] = acc * 2.0 / (double)(D + 1);
    }
    c[0] *= 0.5;
}

// levels the ReLU consumes
u32 relu_depth(double beta, u32 D) { return fheon::cheb_depth(D) + (beta > 1.0 ? 1 : 0); }

int check_args(fheon_ctx *ctx, double beta, u32 D, u32 level)
{
    if (!(beta > 0.0) || !std::isfinite(beta) || D < 1 || D > 1023 || level > ctx->L)
        return fail(ctx, FHEON_ERR_ARG, "relu: beta > 0, 1 <= degree <= 1023, level <= L");
    if (level <= relu_depth(beta, D))
        return fail(ctx, FHEON_ERR_LEVEL, "relu: needs level > %u, got %u", relu_depth(beta, D), level);
    return FHEON_OK;
}

} // namespace

namespace fheon {

// Baby-step/giant-step (Paterson-Stockmeyer) shape of a degree-D series:
// k = 2^ceil(log2(D+1)/2) babies T_1..T_k, m giants T_k, T_2k, .., T_{k 2^(m-1)}
// with D < k 2^m.
void ps_params(u32 D, u32 &k, u32 &m)
{
    u32 b = 0;
    while ((1ull << (2 * b)) < (u64)D + 1) b++; // 2b >= log2(D+1)
    k = 1u << b;
    m = 0;
    while ((u64)k << m <= D) m++;
}

namespace {
// depth of each baby (levels below T_1) and of each giant
struct PsShape {
    u32 k = 0, m = 0;
    std::vector<u32> dep; // [1..min(k, D)]
    std::vector<u32> gd;  // [0..m-1]
};
PsShape ps_shape(u32 D)
{
    PsShape P;
    ps_params(D, P.k, P.m);
    const u32 kb = std::min(P.k, D);
    P.dep.assign(kb + 1, 0);
    for (u32 d = 2; d <= kb; d++) P.dep[d] = std::max(P.dep[d - d / 2], P.dep[d / 2]) + 1;
    if (P.m) P.gd.push_back(P.dep[P.k]);
    for (u32 j = 1; j < P.m; j++) P.gd.push_back(P.gd.back() + 1);
    return P;
}
u32 ps_depth_of(const PsShape &P, u32 deg, u32 j)
{
    if (j == 0) {
        u32 d = 0;
        for (u32 i = 1; i <= std::max(deg, 1u); i++) d = std::max(d, P.dep[i]);
        return d + 1;
    }
    const u32 g = P.k << (j - 1);
    if (deg < g) return ps_depth_of(P, deg, j - 1);
    return std::max(std::max(ps_depth_of(P, deg - g, j - 1), P.gd[j - 1]) + 1, ps_depth_of(P, g - 1, j - 1));
}

// p = r + q T_g for a series of degree < 2g (2 T_g T_j = T_{g+j} + T_{g-j}):
// q_0 = c_g, q_j = 2 c_{g+j}; r_i = c_i (i < g) less c_{g+j} at i = g - j
void cheb_split(const std::vector<double> &c, u32 g, std::vector<double> &q, std::vector<double> &r)
{
    const u32 deg = (u32)c.size() - 1;
    q.assign(1, c[g]);
    for (u32 j = 1; j + g <= deg; j++) q.push_back(2.0 * c[g + j]);
    r.assign(c.begin(), c.begin() + g);
    for (u32 j = 1; j + g <= deg; j++) r[g - j] = r[g - j] - c[g + j];
}

// the tree of one series over `n` parts in lockstep (the same coefficients
// on n inputs): every product of a step goes to the device as one batch
struct PsEval {
    fheon_ctx *ctx;
    std::vector<std::vector<fheon_ct *> *> works;
    u32 n, k, m, top;                           // top: next free working ciphertext
    std::vector<std::vector<fheon_ct *>> T, G;  // [part] babies [1..], giants [0..m-1]
    PlanKeep *keep;

    u32 leaf_level(u32 p, u32 deg) const
    {
        u32 lv = T[p][1]->level;
        for (u32 i = 1; i <= std::max(deg, 1u); i++) lv = std::min(lv, T[p][i]->level);
        return lv - 1;
    }
    u32 out_level(u32 p, u32 deg, u32 j) const
    {
        if (j == 0) return leaf_level(p, deg);
        const u32 g = k << (j - 1);
        if (deg < g) return out_level(p, deg, j - 1);
        return std::min(std::min(out_level(p, deg - g, j - 1), G[p][j - 1]->level) - 1, out_level(p, g - 1, j - 1));
    }
    // sum_i c_i T_i of every part, landing on scale St[p], into out[p]
    int ev(const std::vector<double> &c, u32 j, const std::vector<double> &St, const std::vector<fheon_ct *> &out)
    {
        const u32 deg = (u32)c.size() - 1, N = ctx->N;
        int rc;
        if (j == 0) {
            for (u32 p = 0; p < n; p++) {
                const u32 lv = leaf_level(p, deg) + 1, nt = std::max(deg, 1u);
                const double q = (double)ctx->mod[lv - 1];
                std::vector<const u64 *> src(nt);
                std::vector<u64> stride(nt);
                std::vector<int64_t> K(nt);
                for (u32 i = 1; i <= nt; i++) {
                    const double ci = i <= deg ? c[i] : 0.0;
                    if (!round_int(((ci * St[p]) * q) / T[p][i]->scale, &K[i - 1]))
                        return fail(ctx, FHEON_ERR_ARG, "chebyshev: coefficient factor out of range");
                    src[i - 1] = T[p][i]->c0();
                    stride[i - 1] = (u64)T[p][i]->level * N;
                }
                if ((rc = ct_reshape(ctx, out[p], lv))) return rc;
                FHEON_CUDA(ctx, k_lincomb(ctx, src.data(), stride.data(), K.data(), nt, out[p]->c0(), lv));
                out[p]->scale = St[p] * q; // the sum's scale before the rescale (metadata)
                if ((rc = fheon_rescale(ctx, out[p], out[p]))) return rc;
                out[p]->scale = St[p];
                if ((rc = fheon_add_const(ctx, out[p], c[0], out[p]))) return rc;
            }
            return FHEON_OK;
        }
        const u32 g = k << (j - 1);
        if (deg < g) return ev(c, j - 1, St, out);
        std::vector<double> cq, cr;
        cheb_split(c, g, cq, cr);
        if (top + 2 > works[0]->size()) return fail(ctx, FHEON_ERR_ARG, "chebyshev: working set exhausted");
        std::vector<fheon_ct *> tq(n), tr(n);
        std::vector<double> Sq(n);
        std::vector<u32> lp(n);
        for (u32 p = 0; p < n; p++) {
            tq[p] = (*works[p])[top];
            tr[p] = (*works[p])[top + 1];
            lp[p] = std::min(out_level(p, (u32)cq.size() - 1, j - 1), G[p][j - 1]->level);
            Sq[p] = (St[p] * (double)ctx->mod[lp[p] - 1]) / G[p][j - 1]->scale;
        }
        top += 2;
        if ((rc = ev(cq, j - 1, Sq, tq))) return rc;
        std::vector<RelinItem> items(n);
        for (u32 p = 0; p < n; p++) items[p] = RelinItem{tq[p], G[p][j - 1], lp[p], false, out[p]};
        if ((rc = mul_relin_many(ctx, items.data(), n, keep))) return rc;
        for (u32 p = 0; p < n; p++) {
            if ((rc = fheon_rescale(ctx, out[p], out[p]))) return rc;
            out[p]->scale = St[p];
        }
        if ((rc = ev(cr, j - 1, St, tr))) return rc;
        for (u32 p = 0; p < n; p++) {
            const u32 lo = std::min(out[p]->level, tr[p]->level);
            if (tr[p]->level > lo && (rc = fheon_drop_level(ctx, tr[p], lo, tr[p]))) return rc;
            if (out[p]->level > lo && (rc = fheon_drop_level(ctx, out[p], lo, out[p]))) return rc;
            if ((rc = fheon_add(ctx, tr[p], out[p], out[p]))) return rc;
        }
        top -= 2;
        return FHEON_OK;
    }
};
} // namespace

u32 cheb_depth(u32 D)
{
    const PsShape P = ps_shape(D);
    return ps_depth_of(P, D, P.m);
}

int cheb_work(fheon_ctx *ctx, std::vector<fheon_ct *> &work, u32 D, u32 level, double scale)
{
    // T_1 .. T_k (index d), the giants, two per level of the tree and two
    // temporaries: nothing is allocated after the first application
    u32 k, m;
    ps_params(D, k, m);
    const size_t need = (size_t)std::min(k, D) + m + 2 * (size_t)m + 4;
    if (work.size() < need) work.resize(need, nullptr);
    for (fheon_ct *&c : work) {
        int rc;
        if (!c && (rc = fheon_ct_create(ctx, level, scale, &c))) return rc;
    }
    return FHEON_OK;
}

int cheb_series_many(fheon_ctx *ctx, const std::vector<double> &coeffs, std::vector<fheon_ct *> *const *works, u32 n,
                     fheon_ct *const *outs, PlanKeep *keep)
{
    const u32 D = (u32)coeffs.size() - 1, N = ctx->N;
    u32 k, m;
    ps_params(D, k, m);
    const u32 kb = std::min(k, D);
    int rc;
    std::vector<RelinItem> items(n);
    // babies: operands at a higher level are read in place (their lowest
    // limbs), and the factor 2 of 2 T_a T_b is applied inside the tensor
    for (u32 d = 2; d <= kb; d++) {
        const u32 h = d / 2;
        for (u32 p = 0; p < n; p++) {
            fheon_ct **T = works[p]->data();
            fheon_ct *A = T[d - h], *B = T[h]; // d even: T_h, T_h; odd: T_h+1, T_h
            items[p] = RelinItem{A, B, std::min(A->level, B->level), true, T[d]}; // scale S = s_a s_b
        }
        if ((rc = mul_relin_many(ctx, items.data(), n, keep))) return rc;
        for (u32 p = 0; p < n; p++) {
            fheon_ct **T = works[p]->data();
            const u32 lv = items[p].level;
            if (d % 2 == 1) {
                // - T_1 at scale S joins the product before the shared rescale
                fheon_ct *t1 = (*works[p])[kb + m + 1];
                int64_t K;
                if (!round_int((-1.0 * T[d]->scale) / T[1]->scale, &K))
                    return fail(ctx, FHEON_ERR_ARG, "chebyshev: constant");
                if ((rc = ct_reshape(ctx, t1, lv))) return rc;
                FHEON_CUDA(ctx, k_mul_int(ctx, T[1]->c0(), K, t1->c0(), lv, 2, (u64)T[1]->level * N));
                FHEON_CUDA(ctx, k_add(ctx, T[d]->c0(), t1->c0(), T[d]->c0(), lv, 2));
            }
            if ((rc = fheon_rescale(ctx, T[d], T[d]))) return rc;
            if (d % 2 == 0 && (rc = fheon_add_const(ctx, T[d], -1.0, T[d]))) return rc;
        }
    }
    // giants: G_0 = T_k, G_j = 2 G_j-1^2 - 1
    PsEval E{ctx, std::vector<std::vector<fheon_ct *> *>(works, works + n), n, k, m, kb + m + 2, {}, {}, keep};
    E.T.resize(n);
    E.G.resize(n);
    for (u32 p = 0; p < n; p++) {
        E.T[p].assign(works[p]->begin(), works[p]->begin() + kb + 1);
        if (m) E.G[p].push_back((*works[p])[k]);
    }
    for (u32 j = 1; j < m; j++) {
        for (u32 p = 0; p < n; p++) {
            fheon_ct *A = E.G[p].back();
            items[p] = RelinItem{A, A, A->level, true, (*works[p])[kb + j]};
        }
        if ((rc = mul_relin_many(ctx, items.data(), n, keep))) return rc;
        for (u32 p = 0; p < n; p++) {
            fheon_ct *Gj = (*works[p])[kb + j];
            if ((rc = fheon_rescale(ctx, Gj, Gj))) return rc;
            if ((rc = fheon_add_const(ctx, Gj, -1.0, Gj))) return rc;
            E.G[p].push_back(Gj);
        }
    }
    std::vector<double> St(n);
    for (u32 p = 0; p < n; p++) St[p] = (*works[p])[1]->scale;
    return E.ev(coeffs, m, St, std::vector<fheon_ct *>(outs, outs + n));
}

int cheb_series(fheon_ctx *ctx, const std::vector<double> &coeffs, std::vector<fheon_ct *> &work, fheon_ct *out,
                PlanKeep *keep)
{
    std::vector<fheon_ct *> *w = &work;
    return cheb_series_many(ctx, coeffs, &w, 1, &out, keep);
}

int relu_apply_batch(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins, u32 n, fheon_ct *const *outs)
{
    if (n == 1) return fheon_relu_apply(ctx, ly, ins[0], outs[0]);
    const u32 D = ly->degree;
    int rc;
    if (ly->sets.size() < n) ly->sets.resize(n);
    std::vector<std::vector<fheon_ct *> *> works(n);
    for (u32 p = 0; p < n; p++) {
        const fheon_ct *in = ins[p];
        if (in->level != ly->level) return fail(ctx, FHEON_ERR_LEVEL, "relu expects level %u, got %u", ly->level, in->level);
        if ((rc = cheb_work(ctx, ly->sets[p], D, ly->level, in->scale))) return rc;
        fheon_ct *T1 = ly->sets[p][1];
        if (ly->beta > 1.0) {
            if ((rc = fheon_mul_plain(ctx, in, ly->mask, T1))) return rc;
            if ((rc = fheon_rescale(ctx, T1, T1))) return rc;
            T1->scale = in->scale;
        } else if ((rc = fheon_drop_level(ctx, in, in->level, T1))) {
            return rc;
        }
        works[p] = &ly->sets[p];
    }
    return cheb_series_many(ctx, ly->coeffs, works.data(), n, outs, ly->collect);
}

} // namespace fheon

extern "C" {

uint32_t fheon_cheb_depth(uint32_t degree) { return degree < 1 || degree > 1023 ? 0 : cheb_depth(degree); }

int fheon_relu_coeffs(double beta, uint32_t degree, double *out)
{
    if (!out || !(beta > 0.0) || degree < 1 || degree > 1023) return FHEON_ERR_ARG;
    std::vector<double> c;
    relu_cheb(beta, degree, c);
    for (u32 d = 0; d <= degree; d++) out[d] = c[d];
    return FHEON_OK;
}

int fheon_relu_prepare_plain(fheon_ctx *ctx, double beta, uint32_t degree, const fheon_pt *mask, uint32_t level,
                             fheon_layer **out)
{
    if (!ctx || !out) return FHEON_ERR_ARG;
    int rc = check_args(ctx, beta, degree, level);
    if (rc) return rc;
    if (beta > 1.0 && (!mask || mask->level < level))
        return fail(ctx, FHEON_ERR_ARG, "relu: beta > 1 needs a mask plaintext at level >= %u", level);
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_RELU;
    ly->beta = beta;
    ly->degree = degree;
    ly->level = level;
    relu_cheb(beta, degree, ly->coeffs);
    ly->mask = beta > 1.0 ? const_cast<fheon_pt *>(mask) : nullptr;
    ly->own_mask = false;
    *out = ly.release();
    return FHEON_OK;
}

int fheon_relu_prepare(fheon_ctx *ctx, double beta, uint32_t degree, uint32_t n, uint32_t level, fheon_layer **out)
{
    if (!ctx || !out || n > ctx->N / 2) return FHEON_ERR_ARG;
    int rc = check_args(ctx, beta, degree, level);
    if (rc) return rc;
    fheon_pt *mask = nullptr;
    if (beta > 1.0) {
        // GenerateScaleMask(beta, n): 1/beta in the first n slots, at scale q_{level-1}
        std::vector<double> v(ctx->N / 2, 0.0);
        for (u32 i = 0; i < n; i++) v[i] = 1.0 / beta;
        if ((rc = fheon_encode_plain(ctx, v.data(), nullptr, ctx->N / 2, level, (double)ctx->mod[level - 1], &mask)))
            return rc;
    }
    rc = fheon_relu_prepare_plain(ctx, beta, degree, mask, level, out);
    if (rc) {
        fheon_pt_destroy(mask);
        return rc;
    }
    (*out)->own_mask = true;
    return FHEON_OK;
}

int fheon_cheb_prepare(fheon_ctx *ctx, const double *coeffs, uint32_t degree, uint32_t level, fheon_layer **out)
{
    if (!ctx || !coeffs || !out) return FHEON_ERR_ARG;
    if (degree < 1 || degree > 1023 || level > ctx->L)
        return fail(ctx, FHEON_ERR_ARG, "series: degree in [1, 1023] and level <= L");
    if (level <= cheb_depth(degree))
        return fail(ctx, FHEON_ERR_LEVEL, "series: needs level > %u, got %u", cheb_depth(degree), level);
    std::unique_ptr<fheon_layer> ly(new fheon_layer());
    ly->kind = LAYER_RELU;
    ly->beta = 1.0; // no mask: the input is the series' variable
    ly->degree = degree;
    ly->level = level;
    ly->coeffs.assign(coeffs, coeffs + degree + 1);
    *out = ly.release();
    return FHEON_OK;
}

int fheon_relu_apply(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !ly || !in || !out || ly->kind != LAYER_RELU) return FHEON_ERR_ARG;
    if (in->level != ly->level) return fail(ctx, FHEON_ERR_LEVEL, "relu expects level %u, got %u", ly->level, in->level);
    if (out == in) return fail(ctx, FHEON_ERR_ARG, "relu output must not alias its input");
    const u32 D = ly->degree;
    const double s0 = in->scale;
    int rc;
    if ((rc = cheb_work(ctx, ly->rot, D, ly->level, s0))) return rc;
    fheon_ct *T1 = ly->rot[1];
    // v = x * mask, rescaled (scale q_{l-1} of the mask cancels)
    if (ly->beta > 1.0) {
        if ((rc = fheon_mul_plain(ctx, in, ly->mask, T1))) return rc;
        if ((rc = fheon_rescale(ctx, T1, T1))) return rc;
        T1->scale = s0;
    } else if ((rc = fheon_drop_level(ctx, in, in->level, T1))) {
        return rc;
    }
    return cheb_series(ctx, ly->coeffs, ly->rot, out, ly->collect);
}

int fheon_relu_approx(fheon_ctx *ctx, const fheon_ct *ct, double beta, uint32_t degree, uint32_t n, fheon_ct *out)
{
    if (!ctx || !ct) return FHEON_ERR_ARG;
    fheon_layer *ly = nullptr;
    int rc = fheon_relu_prepare(ctx, beta, degree, n, ct->level, &ly);
    if (rc) return rc;
    rc = fheon_relu_apply(ctx, ly, ct, out);
    fheon_layer_destroy(ly);
    return rc;
}

} // extern "C"
