// relu.cu -- FHEON's secure ReLU (paper Sec. 4.6, Alg. 4) as host
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

u32 ceil_log2(u32 x)
{
    u32 r = 0;
    while ((1u << r) < x) r++;
    return r;
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

struct PsEval {
    fheon_ctx *ctx;
    std::vector<fheon_ct *> &work;
    u32 k, m, top;                    // top: next free working ciphertext
    std::vector<fheon_ct *> T, G;     // babies [1..], giants [0..m-1]

    u32 leaf_level(u32 deg) const
    {
        u32 lv = T[1]->level;
        for (u32 i = 1; i <= std::max(deg, 1u); i++) lv = std::min(lv, T[i]->level);
        return lv - 1;
    }
    u32 out_level(u32 deg, u32 j) const
    {
        if (j == 0) return leaf_level(deg);
        const u32 g = k << (j - 1);
        if (deg < g) return out_level(deg, j - 1);
        return std::min(std::min(out_level(deg - g, j - 1), G[j - 1]->level) - 1, out_level(g - 1, j - 1));
    }
    // sum_i c_i T_i landing on scale St, into `out`
    int ev(const std::vector<double> &c, u32 j, double St, fheon_ct *out)
    {
        const u32 deg = (u32)c.size() - 1, N = ctx->N;
        int rc;
        if (j == 0) {
            const u32 lv = leaf_level(deg) + 1, n = std::max(deg, 1u);
            const double q = (double)ctx->mod[lv - 1];
            std::vector<const u64 *> src(n);
            std::vector<u64> stride(n);
            std::vector<int64_t> K(n);
            for (u32 i = 1; i <= n; i++) {
                const double ci = i <= deg ? c[i] : 0.0;
                if (!round_int(((ci * St) * q) / T[i]->scale, &K[i - 1]))
                    return fail(ctx, FHEON_ERR_ARG, "chebyshev: coefficient factor out of range");
                src[i - 1] = T[i]->c0();
                stride[i - 1] = (u64)T[i]->level * N;
            }
            if ((rc = ct_reshape(ctx, out, lv))) return rc;
            FHEON_CUDA(ctx, k_lincomb(ctx, src.data(), stride.data(), K.data(), n, out->c0(), lv));
            out->scale = St * q; // the sum's scale before the rescale (metadata)
            if ((rc = fheon_rescale(ctx, out, out))) return rc;
            out->scale = St;
            return fheon_add_const(ctx, out, c[0], out);
        }
        const u32 g = k << (j - 1);
        if (deg < g) return ev(c, j - 1, St, out);
        std::vector<double> cq, cr;
        cheb_split(c, g, cq, cr);
        const fheon_ct *Gc = G[j - 1];
        const u32 lp = std::min(out_level((u32)cq.size() - 1, j - 1), Gc->level);
        if (top + 2 > work.size()) return fail(ctx, FHEON_ERR_ARG, "chebyshev: working set exhausted");
        fheon_ct *tq = work[top], *tr = work[top + 1];
        top += 2;
        if ((rc = ev(cq, j - 1, (St * (double)ctx->mod[lp - 1]) / Gc->scale, tq))) return rc;
        if ((rc = mul_relin_at(ctx, tq, Gc, lp, false, out))) return rc;
        if ((rc = fheon_rescale(ctx, out, out))) return rc;
        out->scale = St;
        if ((rc = ev(cr, j - 1, St, tr))) return rc;
        const u32 lo = std::min(out->level, tr->level);
        if (tr->level > lo && (rc = fheon_drop_level(ctx, tr, lo, tr))) return rc;
        if (out->level > lo && (rc = fheon_drop_level(ctx, out, lo, out))) return rc;
        if ((rc = fheon_add(ctx, tr, out, out))) return rc;
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

int cheb_series(fheon_ctx *ctx, const std::vector<double> &coeffs, std::vector<fheon_ct *> &work, fheon_ct *out)
{
    const u32 D = (u32)coeffs.size() - 1, N = ctx->N;
    u32 k, m;
    ps_params(D, k, m);
    const u32 kb = std::min(k, D);
    fheon_ct **T = work.data();
    fheon_ct *t1 = work[kb + m + 1];
    int rc;
    // babies: operands at a higher level are read in place (their lowest
    // limbs), and the factor 2 of 2 T_a T_b is applied inside the tensor
    for (u32 d = 2; d <= kb; d++) {
        const u32 h = d / 2;
        fheon_ct *A = T[d - h], *B = T[h]; // d even: T_h, T_h; odd: T_h+1, T_h
        const u32 lv = A->level < B->level ? A->level : B->level;
        if ((rc = mul_relin_at(ctx, A, B, lv, true, T[d]))) return rc; // scale S = s_a s_b
        if (d % 2 == 1) {
            // - T_1 at scale S joins the product before the shared rescale
            int64_t K;
            if (!round_int((-1.0 * T[d]->scale) / T[1]->scale, &K)) return fail(ctx, FHEON_ERR_ARG, "chebyshev: constant");
            if ((rc = ct_reshape(ctx, t1, lv))) return rc;
            FHEON_CUDA(ctx, k_mul_int(ctx, T[1]->c0(), K, t1->c0(), lv, 2, (u64)T[1]->level * N));
            FHEON_CUDA(ctx, k_add(ctx, T[d]->c0(), t1->c0(), T[d]->c0(), lv, 2));
        }
        if ((rc = fheon_rescale(ctx, T[d], T[d]))) return rc;
        if (d % 2 == 0 && (rc = fheon_add_const(ctx, T[d], -1.0, T[d]))) return rc;
    }
    // giants: G_0 = T_k, G_j = 2 G_j-1^2 - 1
    PsEval E{ctx, work, k, m, kb + m + 2, {}, {}};
    E.T.assign(T, T + kb + 1);
    if (m) E.G.push_back(T[k]);
    for (u32 j = 1; j < m; j++) {
        fheon_ct *A = E.G.back(), *Gj = work[kb + j];
        if ((rc = mul_relin_at(ctx, A, A, A->level, true, Gj))) return rc;
        if ((rc = fheon_rescale(ctx, Gj, Gj))) return rc;
        if ((rc = fheon_add_const(ctx, Gj, -1.0, Gj))) return rc;
        E.G.push_back(Gj);
    }
    return E.ev(coeffs, m, T[1]->scale, out);
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
    return cheb_series(ctx, ly->coeffs, ly->rot, out);
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
