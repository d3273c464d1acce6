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
// ceil(log2 D) + 1, + 1 for the mask):
//   T_1 = v; T_2h = 2 T_h^2 - 1; T_2h+1 = 2 T_h+1 T_h - T_1,
// each product taken at the lower operand's level with relinearisation and
// rescaled; T_1 is brought to the product's level and exact scale by a
// rescaled constant product (c = -1).  Then every c_d T_d (d >= 1) is
// rescaled onto the input's scale at one common level, the terms are summed
// in order of d, and c_0 is added.  The output has the input's scale.
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

u32 cheb_depth(u32 D) { return ceil_log2(D) + 1; }

int cheb_work(fheon_ctx *ctx, std::vector<fheon_ct *> &work, u32 D, u32 level, double scale)
{
    // T_1 .. T_D (index d), two temporaries and the sum: nothing is allocated
    // after the first application
    if (work.size() != D + 4) work.resize(D + 4, nullptr);
    for (fheon_ct *&c : work) {
        int rc;
        if (!c && (rc = fheon_ct_create(ctx, level, scale, &c))) return rc;
    }
    return FHEON_OK;
}

int cheb_series(fheon_ctx *ctx, const std::vector<double> &coeffs, std::vector<fheon_ct *> &work, fheon_ct *out)
{
    const u32 D = (u32)coeffs.size() - 1, N = ctx->N;
    fheon_ct **T = work.data();
    fheon_ct *t1 = work[D + 2], *y = work[D + 3];
    const double s0 = T[1]->scale;
    int rc;
    // operands at a higher level are read in place (their lowest limbs), and
    // the factor 2 of 2 T_a T_b is applied inside the tensor
    for (u32 d = 2; d <= D; d++) {
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
    u32 lstar = T[1]->level;
    for (u32 d = 1; d <= D; d++) lstar = T[d]->level < lstar ? T[d]->level : lstar;
    lstar -= 1;
    // y = sum_d K_d T_d at level lstar + 1 in one pass, rescaled once onto s0
    std::vector<const u64 *> src(D);
    std::vector<u64> stride(D);
    std::vector<int64_t> K(D);
    const double q = (double)ctx->mod[lstar];
    for (u32 d = 1; d <= D; d++) {
        if (!round_int(((coeffs[d] * s0) * q) / T[d]->scale, &K[d - 1]))
            return fail(ctx, FHEON_ERR_ARG, "chebyshev: coefficient factor out of range");
        src[d - 1] = T[d]->c0();
        stride[d - 1] = (u64)T[d]->level * N;
    }
    if ((rc = ct_reshape(ctx, y, lstar + 1))) return rc;
    FHEON_CUDA(ctx, k_lincomb(ctx, src.data(), stride.data(), K.data(), D, y->c0(), lstar + 1));
    y->scale = s0 * q; // the sum's scale before the rescale (metadata)
    if ((rc = fheon_rescale(ctx, y, y))) return rc;
    y->scale = s0;
    return fheon_add_const(ctx, y, coeffs[0], out);
}

} // namespace fheon

extern "C" {

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
    if (!ctx || !coeffs || !out || degree < 1 || degree > 1023 || level > ctx->L) return FHEON_ERR_ARG;
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
