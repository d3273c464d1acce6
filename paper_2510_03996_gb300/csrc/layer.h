// layer.h -- the state behind a fheon_layer handle: one prepared layer of an
// encrypted network (conv, approximate ReLU), its plaintexts, working
// ciphertexts and captured graphs.
#pragma once
#include <complex>
#include <map>
#include <set>
#include <vector>

#include "internal.h"

// kinds of layer behind the one opaque handle
enum LayerKind : u32 { LAYER_CONV = 0, LAYER_RELU = 1, LAYER_LINEAR = 2, LAYER_FC = 3, LAYER_BOOT = 4 };

struct fheon_layer {
    u32 kind = LAYER_CONV;
    u32 in_ch = 0, k = 0, H = 0, W = 0, level = 0;
    // approximate ReLU (Alg. 4): beta, degree, Chebyshev coefficients c_0..c_D;
    // `mask` holds the 1/beta scale mask when beta > 1
    double beta = 1.0;
    u32 degree = 0;
    std::vector<double> coeffs;
    // rotation-sum layer: tap steps r_t (hoisted from the input), group shifts
    // s_g, plaintexts [g][t] (null: no product); FC: weight and placement
    // plaintexts of each output neuron, the slots summed over
    std::vector<int32_t> r, s;
    std::vector<int32_t> fold; // rotation-sum layer: the input first becomes sum_c Rot_{fold[c]}(in)
    std::vector<fheon_pt *> pts, fw, fe;   // views
    std::vector<fheon_pt *> pt_store;       // the plaintexts the layer owns
    u32 nslots = 0;
    fheon_map in_map{}, out_map{};
    std::vector<fheon_pt *> taps; // k*k, row-major (di, dj)
    fheon_pt *mask = nullptr;     // conv with C > 1: block-0 mask at level-1; ReLU: the 1/beta mask
    bool own_mask = true;
    fheon_pt *bias = nullptr;     // at the output level
    std::vector<bool> owned;      // which of taps are owned by the layer
    bool own_bias = false;
    // bootstrapping: the CoeffToSlot then SlotToCoeff levels (rotation-sum
    // layers; owned when own_subs), EvalMod's series in `coeffs` with range K
    // and r doublings, the scale inputs must have, X^(N/2) at the two levels
    // it multiplies at, and the output's level and scale
    std::vector<fheon_layer *> subs;
    u32 ncts = 0, boot_K = 0, boot_r = 0;
    bool own_subs = false;
    double in_scale = 0, out_scale = 0;
    u32 out_level = 0;
    fheon_pt *mono[2] = {nullptr, nullptr};
    // sparse bootstrap: the message slots n_s (0: every slot) and the input
    // mask of slots [0, n_s) at level 2, scale q_1 (owned unless set by the caller)
    u32 boot_ns = 0;
    bool boot_unmasked = false; // inputs zero outside [0, n_s): no mask, level 1 taken
    const fheon_pt *boot_mask = nullptr;
    bool own_boot_mask = false;
    mutable std::vector<fheon_ct *> cheb2; // the second part's series working set
    mutable std::vector<std::vector<fheon_ct *>> sets; // ReLU on a batch: one working set per input
    // bootstrapping a batch: per input, its 10 working ciphertexts and the two
    // series working sets (the single-input path uses work, rot and cheb2)
    struct BootSet {
        std::vector<fheon_ct *> w, re, im;
    };
    mutable std::vector<BootSet> bsets;
    // working ciphertexts (the k^2 - 1 tap rotations, then accumulators), made
    // on the first application and reused, so that later applications (and
    // their graph capture) allocate nothing
    mutable std::vector<fheon_ct *> rot;
    mutable std::vector<fheon_ct *> work, fwork;
    mutable fheon_ct *tmp[3] = {nullptr, nullptr, nullptr};
    // captured applications, keyed by the buffers the captured launches use;
    // `keep` holds the device rotation plans those launches read
    struct Graph {
        const void *in, *out, *ws;
        u32 level;
        double scale;           // the input's scale (captured constants depend on it)
        u32 out_level;          // the output's metadata the captured run set
        double out_scale;
        cudaGraphExec_t exec;
        fheon::PlanKeep keep;
    };
    mutable std::vector<Graph> graphs;
    mutable fheon::PlanKeep *collect = nullptr; // set while an application is captured
    ~fheon_layer()
    {
        for (size_t i = 0; i < taps.size(); i++)
            if (owned[i]) fheon_pt_destroy(taps[i]);
        if (own_mask) fheon_pt_destroy(mask);
        if (own_bias) fheon_pt_destroy(bias);
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        for (fheon_ct *c : tmp) fheon_ct_destroy(c);
        for (fheon_ct *c : rot) fheon_ct_destroy(c);
        for (fheon_ct *c : work) fheon_ct_destroy(c);
        for (fheon_ct *c : fwork) fheon_ct_destroy(c);
        for (fheon_pt *p : pt_store) fheon_pt_destroy(p);
        if (own_subs)
            for (fheon_layer *l : subs) delete l;
        for (fheon_pt *p : mono) fheon_pt_destroy(p);
        if (own_boot_mask) fheon_pt_destroy(const_cast<fheon_pt *>(boot_mask));
        for (fheon_ct *c : cheb2) fheon_ct_destroy(c);
        for (auto &v : sets)
            for (fheon_ct *c : v) fheon_ct_destroy(c);
        for (auto &b : bsets)
            for (auto *v : {&b.w, &b.re, &b.im})
                for (fheon_ct *c : *v) fheon_ct_destroy(c);
    }
};

namespace fheon {
// Chebyshev series (relu.cu): `work` holds the working ciphertexts
// (cheb_work makes them); work[1] = T_1 on entry, at the series' input
// scale; out = sum_d c_d T_d at that scale, cheb_depth(D) levels below
int cheb_work(fheon_ctx *ctx, std::vector<fheon_ct *> &work, u32 D, u32 level, double scale);
int cheb_series(fheon_ctx *ctx, const std::vector<double> &coeffs, std::vector<fheon_ct *> &work, fheon_ct *out,
                PlanKeep *keep = nullptr);
// the same series on n inputs in lockstep (works[p][1] = T_1 of part p), the
// products of each step in one batch; each output is the one cheb_series gives
int cheb_series_many(fheon_ctx *ctx, const std::vector<double> &coeffs, std::vector<fheon_ct *> *const *works, u32 n,
                     fheon_ct *const *outs, PlanKeep *keep = nullptr);
u32 cheb_depth(u32 D);
// slot diagonals of a linear map on n slots: out = sum_o d_o * Rot_o(in)
using cd = std::complex<double>;
using Diags = std::map<u32, std::vector<cd>>; // offset mod n -> diagonal
// BSGS form of sum_o d_o Rot_o: offsets k * stride (k centred in (-M/2, M/2],
// M = n / stride) split as k = c bs + t, 0 <= t < bs:
//   out = sum_c Rot_{G_c}( sum_t Rot_{-G_c}(d_k) Rot_{t stride}(in) ),  G_c = c bs stride.
// bs = `baby`, else the power of two with the fewest rotations (ties: larger).
struct Bsgs {
    std::vector<int32_t> r, s;
    std::vector<std::vector<cd>> vals; // [g * r.size() + t], empty = no product
};
Bsgs bsgs_plan(const Diags &D, u32 n, u32 stride, u32 baby);
// the split alone, from the nonzero offsets: k = o / stride centred in
// (-M/2, M/2] (bsgs_offsets), then the baby-step size bs over b = 1, 2, ..
// <= M (fewest rotations, ties: the larger), the baby steps ts and giant
// steps cs; r = ts * stride, s = cs * bs * stride
std::set<int64_t> bsgs_offsets(const std::set<u32> &offsets, u32 n, u32 stride);
void bsgs_split(const std::set<int64_t> &ks, int64_t M, u32 baby, int64_t &bs, std::set<int64_t> &ts,
                std::set<int64_t> &cs);
// baby steps B of a C -> F convolution with a k x k kernel: the B minimising
// B k^2 - 1 + 2 ceil((C + F - 1) / B) (hoisted tap rotations, plus the giant
// steps at twice a hoisted rotation's cost), the smaller on ties
u32 conv_baby(u32 k, u32 C, u32 F);
// rotation steps of the repack layer from map a to map b (the plan of
// fheon_repack_prepare, without encoding it); FHEON_ERR_ARG as that call
int repack_steps(u32 n, const fheon_map &a, const fheon_map &b, std::vector<int32_t> &steps);
// the rotation-sum layer of sum_o (factor d_o) Rot_o at `level`, its
// plaintexts encoded at `pscale` and owned by the layer
int diag_layer(fheon_ctx *ctx, const Diags &M, u32 stride, cd factor, u32 baby, u32 level, double pscale,
               fheon_layer **out);
// the ReLU layer on n inputs, their series in lockstep (relu.cu)
int relu_apply_batch(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins, u32 n, fheon_ct *const *outs);
// bootstrapping (boot.cu)
int boot_apply(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *in, fheon_ct *out);
// n inputs at once: every level, the conjugations, the series and the
// doublings of all of them as batches; each output is the one boot_apply gives
int boot_apply_many(fheon_ctx *ctx, const fheon_layer *ly, const fheon_ct *const *ins, u32 n, fheon_ct *const *outs);
} // namespace fheon
