"""The oracle's pins catch plausible mistakes: each case plants one mistake in
the oracle (a dropped term, a wrong sign, a transposed operand, a wrong index)
and checks that the pin written for that part fails.

C mistakes are planted in a copy of ckks_oracle.c, compiled with the oracle's
own flags into a temporary library that stands in for the oracle's for the
duration of one test; the oracle's source is not touched.  Python mistakes are
planted with monkeypatch.  Every planted mistake runs on the CPU."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import test_oracle_boot as TB
import test_oracle_fheon as TF
import test_oracle_hoisted as TH
import test_oracle_layers as TL
import test_oracle_mult as TM
import test_oracle_paper_layers as TP
import test_oracle_primitives as PR
import test_oracle_relu as TR
import test_oracle_scheme as S
from oracle import _lib
from oracle import boot as B
from oracle import ckks
from oracle import fheon as OF
from oracle import paper_layers as PL
from paper_2510_03996_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ckks_oracle.c")


def _tiny():
    ctx, P = S._ctx("tiny")
    s, se = ctx.keygen_sk()
    return ctx, P, s, se, ctx.keygen_pk(se)


def _tiny4():
    ctx, P, s, se, pk = _tiny()
    return ctx, P, se, pk


# name: (C function holding the site, exact text, planted text, the pin that must fail)
C_PLANTS = {
    "chacha_rotation": ("static void quarter(", "x[d] = rotl32(x[d], 16);", "x[d] = rotl32(x[d], 15);",
                        lambda: PR.test_chacha20_rfc8439_vector()),
    "cdt_variance": ("void oracle_cdt_table(", "(2.0 * sigma * sigma)", "(sigma * sigma)",
                     lambda: PR.test_cdt_table_against_high_precision()),
    "ntt_butterfly_sign": ("static void ntt_fast(", "a[j + t] = submod(U, V, q);", "a[j + t] = addmod(U, V, q);",
                           lambda: PR.test_fast_ntt_equals_definition(6)),
    "ntt_twiddle_order": ("static void ntt_fast(", "u64 S = tw[m + i];", "u64 S = tw[m + (m - 1 - i)];",
                          lambda: PR.test_fast_ntt_equals_definition(6)),
    "automorphism_wrap_sign": ("void oracle_automorph_coeff(", "else out[e - N] = submod(0, a[i] % q, q);",
                               "else out[e - N] = a[i] % q;",
                               lambda: PR.test_automorph_coeff_definition_and_composition()),
    "bconv_missing_inverse": ("void oracle_bconv(", "u64 y = mulmod(in[(size_t)i * N + n], inv, from[i]);",
                              "u64 y = in[(size_t)i * N + n] % from[i]; (void)inv;",
                              lambda: PR.test_bconv_against_exact_crt()),
    "modup_digit_dropped": ("void oracle_modup(",
                            "memcpy(out + (size_t)l * N, x_coeff + (size_t)l * N, sizeof(u64) * N);",
                            "memset(out + (size_t)l * N, 0, sizeof(u64) * N);",
                            lambda: S.test_modup_is_crt_lift_plus_small_multiple(_tiny())),
    "moddown_sign": ("void oracle_moddown(", "mulmod(submod(x_coeff[o], conv[o], q), Pinv, q)",
                     "mulmod(addmod(x_coeff[o], conv[o], q), Pinv, q)",
                     lambda: S.test_moddown_is_floor_division_minus_small(_tiny())),
    "rescale_no_subtraction": ("void oracle_rescale_poly(", "mulmod(submod(x[o], ri[k], q), inv, q)",
                               "mulmod(x[o], inv, q)", lambda: S.test_rescale_is_floor_division(_tiny())),
    "ksk_missing_P": ("void oracle_keygen_ksk(", "addmod(v, mulmod(Pm, sfrom_eval[o], m), m)",
                      "addmod(v, sfrom_eval[o], m)", lambda: S.test_keyswitch_noise_bound(_tiny())),
    "keyswitch_key_components_swapped": ("void oracle_keyswitch(", "(((size_t)j * 2 + b) * nall + mi)",
                                         "(((size_t)j * 2 + (1 - b)) * nall + mi)",
                                         lambda: S.test_rotate_decrypts_to_automorphism(_tiny(), 1)),
    "rotate_c0_dropped": ("void oracle_rotate(", "out[o] = addmod(sc[o], ks[o], c->mod[i]);", "out[o] = ks[o];",
                          lambda: S.test_rotate_decrypts_to_automorphism(_tiny(), 3)),
    "encrypt_message_dropped": ("void oracle_encrypt(", "addmod(addmod(mulmod(V[o], pk[o], q), E0[o], q), M[o], q)",
                                "addmod(mulmod(V[o], pk[o], q), E0[o], q)",
                                lambda: S.test_encrypt_decrypt_noise_bound(_tiny())),
    "encode_truncates": ("int oracle_encode(", "double r = round(v);", "double r = trunc(v);",
                         lambda: S.test_encode_rounds_half_away_from_zero()),
    "encode_conjugated": ("int oracle_encode(", "acc += zr[i] * cs[e] - zi[i] * sn[e];",
                          "acc += zr[i] * cs[e] + zi[i] * sn[e];", lambda: S.test_encode_decode_roundtrip(64)),
    "decode_sign": ("void oracle_decode(", "ai += m[k] * sn[e];", "ai -= m[k] * sn[e];",
                    lambda: S.test_decode_matches_independent_fft_formulation()),
    "tensor_cross_term_dropped": ("void oracle_mul_relin(",
                                  "addmod(mulmod(a[o], b[pl + o], q), mulmod(a[pl + o], b[o], q), q)",
                                  "mulmod(a[o], b[pl + o], q)",
                                  lambda: TM.test_mul_relin_decrypts_to_the_product(_tiny(), 4)),
    "relu_wrong_side": ("void oracle_cheb_coeffs(", "z < 0.0 ? 0.0 : beta * z", "z > 0.0 ? 0.0 : beta * z",
                        lambda: TR.test_coeffs_are_chebyshev_interpolation(1.0, 59)),
    "evalmod_phase_sign": ("void oracle_cos_cheb_coeffs(", "(K * z - 0.25)", "(K * z + 0.25)",
                           lambda: TB.test_evalmod_series_and_doublings()),
    "intt_butterfly_sign": ("static void intt_fast(", "mulmod(submod(U, V, q), S, q)", "mulmod(addmod(U, V, q), S, q)",
                            lambda: PR.test_fast_ntt_equals_definition(6)),
    "psi_not_minimal": ("u64 oracle_min_psi(", "if (cur < best) best = cur;", "if (cur > best) best = cur;",
                        lambda: PR.test_min_psi_brute_force(97, 16)),
    "prime_not_largest": ("int oracle_gen_primes(", "u64 cand = top - ((top - 1) % twoN);",
                          "u64 cand = top - ((top - 1) % twoN) - twoN;",
                          lambda: PR.test_gen_primes_are_the_largest_ntt_primes(13, [60, 40, 40, 60])),
    "ternary_two_values": ("void oracle_sample_ternary(", "% 3) - 1", "% 2) - 1",
                           lambda: PR.test_samplers_statistics()),
    "gauss_index_shifted": ("void oracle_sample_gauss(", "out[n] = k;", "out[n] = k + 1;",
                            lambda: PR.test_samplers_statistics()),
    "uniform_words_swapped": ("void oracle_sample_uniform(", "(((u128)hi << 64) | lo) % q",
                              "(((u128)lo << 64) | hi) % q", lambda: PR.test_samplers_statistics()),
    "automorphism_element_conjugated": ("void oracle_automorph_eval(", "oracle_automorph_coeff(t, N, c->mod[mi], g, t2);",
                                        "oracle_automorph_coeff(t, N, c->mod[mi], 2ull * N - g, t2);",
                                        lambda: S.test_rotate_decrypts_to_automorphism(_tiny(), 1)),
    "hoisted_c0_not_permuted": ("void oracle_rotate_hoisted(", "oracle_automorph_eval(c, ct, level, 0, gs[r], sc0);",
                                "memcpy(sc0, ct, sizeof(u64) * pl);",
                                lambda: TH.test_constant_c1_equals_plain_rotation_for_every_g(_tiny4(), 4)),
    "hoisted_digits_not_permuted": ("void oracle_rotate_hoisted(",
                                    "oracle_automorph_eval(c, ext + j * limbs, level, 1, gs[r], d);",
                                    "memcpy(d, ext + j * limbs, sizeof(u64) * limbs);",
                                    lambda: TH.test_decrypts_to_automorphism_and_differs_from_plain(_tiny4())),
    "decrypt_sign": ("void oracle_decrypt(", "m[o] = addmod(ct[o], mulmod(", "m[o] = submod(ct[o], mulmod(",
                     lambda: S.test_encrypt_decrypt_noise_bound(_tiny())),
    "public_key_sign": ("void oracle_keygen_pk(", "addmod(submod(0, mulmod(a[k], s_eval[(size_t)i * N + k], q), q)",
                        "addmod(mulmod(a[k], s_eval[(size_t)i * N + k], q)",
                        lambda: S.test_public_key_relation(_tiny())),
    "mul_int_sign": ("void oracle_mul_int(", "vm = from_signed(v, q);", "vm = from_signed(-v, q);",
                     lambda: TM.test_mul_int_and_add_int_are_exact(_tiny())),
    "ntt_definition_natural_order": ("void oracle_ntt_def(", "powmod(psi, 2ull * brv(j, logn) + 1, q)",
                                     "powmod(psi, 2ull * j + 1, q)",
                                     lambda: PR.test_ntt_definition_brute_force(97, 16)),
    "schoolbook_wrap_sign": ("void oracle_negacyclic_mul(", "else out[i + j - N] = submod(out[i + j - N], p, q);",
                             "else out[i + j - N] = addmod(out[i + j - N], p, q);",
                             lambda: PR.test_convolution_theorem()),
    "draw_block_counter": ("u64 oracle_draw64(", "(u32)(n / 8)", "(u32)(n / 16)",
                           lambda: PR.test_draw64_is_word_pair_of_block()),
    "secret_key_one_modulus": ("void oracle_keygen_sk(", "midx[i] = i;", "midx[i] = 0;",
                               lambda: S.test_secret_key_is_ternary_and_consistent(_tiny())),
    "mul_plain_c1_skipped": ("void oracle_mul_plain(", "out[b * pl + o] = mulmod(ct[b * pl + o], pt[o], c->mod[i]);",
                             "out[b * pl + o] = b ? ct[b * pl + o] : mulmod(ct[b * pl + o], pt[o], c->mod[i]);",
                             lambda: S.test_add_and_mul_plain_exact(_tiny())),
    "add_subtracts": ("void oracle_add(", "out[o] = addmod(x[o], y[o], c->mod[i]);",
                      "out[o] = submod(x[o], y[o], c->mod[i]);", lambda: S.test_add_and_mul_plain_exact(_tiny())),
    "miller_rabin_one_base": ("int oracle_is_prime(", "for (int i = 0; i < 12; i++) {\n        u64 x",
                              "for (int i = 0; i < 1; i++) {\n        u64 x", lambda: PR.test_is_prime_against_sympy()),
    "add_plain_into_c1": ("void oracle_add_plain(",
                          "out[o] = addmod(ct[o], pt[o], c->mod[i]);\n            out[pl + o] = ct[pl + o];",
                          "out[o] = ct[o];\n            out[pl + o] = addmod(ct[pl + o], pt[o], c->mod[i]);",
                          lambda: S.test_add_and_mul_plain_exact(_tiny())),
    "tensor_d0_dropped": ("void oracle_mul_relin(", "d[o] = mulmod(a[o], b[o], q);", "d[o] = 0;",
                          lambda: TM.test_mul_relin_decrypts_to_the_product(_tiny(), 3)),
    "add_int_into_c1": ("void oracle_add_int(", "out[o] = addmod(ct[o], vm, q);\n            out[pl + o] = ct[pl + o];",
                        "out[o] = ct[o];\n            out[pl + o] = addmod(ct[pl + o], vm, q);",
                        lambda: TM.test_mul_int_and_add_int_are_exact(_tiny())),
}


def plant_c(src, func, old, new):
    """src with `old` replaced by `new` inside the body of the C function whose
    definition starts with `func` (the text must occur there exactly once)."""
    start = src.index(func)
    end = src.index("\n}\n", start)
    body = src[start:end]
    assert body.count(old) == 1, (func, old)
    return src[:start] + body.replace(old, new) + src[end:]


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


def build_mutant(directory, name, source):
    c = os.path.join(str(directory), name + ".c")
    so = os.path.join(str(directory), "lib" + name + ".so")
    with open(c, "w") as f:
        f.write(source)
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-o", so, c, "-lm"], check=True)
    L = ctypes.CDLL(so)
    for fn, (res, args) in _lib._SIGS.items():
        f = getattr(L, fn)
        f.restype = res
        f.argtypes = args
    return L


def test_every_c_site_is_in_the_oracle():
    src = open(SRC).read()
    for name, (func, old, new, _) in C_PLANTS.items():
        assert plant_c(src, func, old, new) != src, name


@pytest.mark.parametrize("name", sorted(C_PLANTS))
def test_planted_c_mistake_fails_its_pin(name, mutant_dir, monkeypatch):
    func, old, new, pin = C_PLANTS[name]
    _lib.lib()  # the oracle's own library is built and loaded first
    L = build_mutant(mutant_dir, name, plant_c(open(SRC).read(), func, old, new))
    monkeypatch.setattr(_lib, "_lib", L)
    with pytest.raises(AssertionError):
        pin()


# ---------------------------------------------------------------- Python plants
def _conjugated_stages(monkeypatch):
    orig = B.stage_diagonals
    monkeypatch.setattr(B, "stage_diagonals",
                        lambda n, h, inverse=False: {o: np.conj(d) for o, d in orig(n, h, inverse).items()})


def _giant_step_rotated_the_wrong_way(monkeypatch):
    orig = B.bsgs_plan

    def bad(diags, n, stride, baby=0):
        r, groups = orig(diags, n, stride, baby)
        return r, [(G, [None if v is None else np.roll(v, -2 * G) for v in vals]) for G, vals in groups]
    monkeypatch.setattr(B, "bsgs_plan", bad)


def _series_remainder_uncorrected(monkeypatch):
    orig = OF.cheb_split
    monkeypatch.setattr(OF, "cheb_split", lambda c, g: (orig(c, g)[0], list(c[:g])))


def _mask_shifted(monkeypatch):
    orig = OF.build_mask
    monkeypatch.setattr(OF, "build_mask", lambda sp, ep, w, m, C: np.roll(orig(sp, ep, w, m, C), 1))


def _kernel_transposed(monkeypatch):
    orig = OF.conv_plan

    def bad(*a, **kw):
        a = list(a)
        a[10] = np.swapaxes(np.asarray(a[10]), 2, 3)
        return orig(*a, **kw)
    monkeypatch.setattr(OF, "conv_plan", bad)


def _repack_shift_reversed(monkeypatch):
    def bad(C, H, W, src, dst, nslots):
        a = OF.map_slots(C, H, W, *src)
        b = OF.map_slots(C, H, W, *dst)
        diags = {}
        for s_, d_ in zip(a, b):
            o = int((d_ - s_) % nslots)  # planted: the shift taken the other way
            diags.setdefault(o, np.zeros(nslots))[int(d_)] = 1.0
        stride = nslots
        for o in diags:
            while stride > 1 and o % stride:
                stride //= 2
        return OF.bsgs_plan(diags, nslots, stride)
    monkeypatch.setattr(OF, "repack_plan", bad)


def _raise_uncentred(monkeypatch):
    def bad(ctx, ct):
        out = np.zeros((2, ctx.L, ctx.N), dtype=np.uint64)
        for b in range(2):
            c = ctx.to_coeff(np.ascontiguousarray(ct[b, :1]), 1)[0].astype(np.int64)  # planted: no centring
            res = np.stack([(c % int(qi)).astype(np.uint64) for qi in ctx.q])
            out[b] = ctx.to_eval(res, ctx.L)
        return out
    monkeypatch.setattr(B, "mod_raise", bad)


def _pool_mask_one_over_k(monkeypatch):
    orig = OF.avgpool_plan

    def bad(C, k, stride, H, W, grid, dil, block, nslots):
        r, groups = orig(C, k, stride, H, W, grid, dil, block, nslots)
        return r, [(G, [None if v is None else v * k for v in vals]) for G, vals in groups]  # 1/k, not 1/k^2
    monkeypatch.setattr(OF, "avgpool_plan", bad)


def _fold_rotated_the_wrong_way(monkeypatch):
    orig = OF.fold_slots
    monkeypatch.setattr(OF, "fold_slots", lambda v, fold: orig(v, [-f for f in fold]))


def _kernel_read_transposed(monkeypatch):
    def bad(x, H, W, C, K, k):
        n = len(x)
        p = (k - 1) // 2
        acc = np.zeros(n)
        for (di, dj) in OF.taps(k):
            vec = np.zeros(n)
            for c in range(C):  # planted: the kernel read at (dj, di)
                vec[c * H * W:(c + 1) * H * W] = K[c, dj + p, di + p] * OF.tap_mask(H, W, 1, di, dj)
            acc += vec * OF.rot_slots(x, di * W + dj)
        tot, cur = acc.copy(), acc
        for _ in range(C - 1):
            cur = OF.rot_slots(cur, H * W)
            tot = tot + cur
        out = np.zeros(n)
        out[:H * W] = tot[:H * W]
        return out
    monkeypatch.setattr(OF, "special_conv_slots", bad)


def _doubling_without_minus_one(monkeypatch):
    def bad(x, K, r, D=B.BOOT_DEGREE):
        c = OF.cheb_eval_fp64(B.evalmod_coeffs(K, r, D), x)
        for _ in range(r):
            c = 2.0 * c * c  # planted: the -1 of cos(2a) = 2 cos(a)^2 - 1 dropped
        return c
    monkeypatch.setattr(B, "evalmod_fp64", bad)


def _stage_groups_reversed(monkeypatch):
    orig = B.stage_groups
    monkeypatch.setattr(B, "stage_groups", lambda logn, levels: list(reversed(orig(logn, levels))))


def _crt_not_centred(monkeypatch):
    def bad(residues, moduli):
        Q = 1
        for q in moduli:
            Q *= int(q)
        out = []
        for k in range(residues.shape[1]):
            x = 0
            for q, row in zip(moduli, residues):
                Qh = Q // int(q)
                x += int(row[k]) * Qh * pow(Qh, -1, int(q))
            out.append(x % Q)  # planted: the lift left in [0, Q), not centred
        return out
    monkeypatch.setattr(ckks, "crt_centered", bad)


def _galois_generator_3(monkeypatch):
    monkeypatch.setattr(ckks, "galois_elt", lambda r, N: pow(3, r % (N // 2), 2 * N))


def _monomial_sign(monkeypatch):
    orig = B.monomial
    monkeypatch.setattr(B, "monomial", lambda ctx, level, sign=1: orig(ctx, level, -sign))


def _copy_factor_conjugated(monkeypatch):
    orig = B.copy_factor
    monkeypatch.setattr(B, "copy_factor", lambda ns, n: np.conj(orig(ns, n)))


def _join_map_swapped(monkeypatch):
    orig = B.join_map

    def bad(ns, n):
        d = orig(ns, n)
        return {0: d[ns % n], ns % n: d[0]}
    monkeypatch.setattr(B, "join_map", bad)


def _trace_skipped(monkeypatch):
    orig = B.mod_raise

    def bad(ctx, ct):
        r = orig(ctx, ct)
        monkeypatch.setattr(B.Plan, "trace_steps", lambda self: [])  # planted: no trace after ModRaise
        return r
    monkeypatch.setattr(B, "mod_raise", bad)


def _rotation_remapped(remap):
    """A paper-form layer that rotates by remap(r) where it means r (a wrong
    shift in one of its steps)."""
    def plant(monkeypatch):
        orig = PL.Counter.rot
        monkeypatch.setattr(PL.Counter, "rot", lambda self, x, r: orig(self, x, remap(r)))
    return plant


@pytest.fixture(scope="module")
def boot_ctx():
    P = synth.params("boot_n12")
    N = 1 << P["logN"]
    L = len(P["qbits"])
    pr = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    ctx = ckks.Ctx(N, pr[:L], pr[L:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    return P, ctx, s, se, ctx.keygen_pk(se), B.Plan(ctx, P["scale"])


PY_PLANTS = {
    "stage_twiddle_conjugated": (_conjugated_stages, lambda bc: TB.test_stages_are_the_slot_transform(16)),
    "giant_step_prerotation_sign": (_giant_step_rotated_the_wrong_way,
                                    lambda bc: TB.test_merged_levels_in_bsgs_form(2)),
    "series_remainder_uncorrected": (_series_remainder_uncorrected, lambda bc: TR.test_series_tree_and_depth()),
    "alg2_mask_shifted": (_mask_shifted, lambda bc: TF.test_build_mask_worked_case()),
    "conv_kernel_transposed": (_kernel_transposed,
                               lambda bc: TL.test_conv_plan_is_the_convolution(1, 3, 3, 0, 6, 8, 1)),
    "special_conv_kernel_transposed": (_kernel_read_transposed,
                                     lambda bc: TF.test_special_conv_slots_equals_fp64_same_conv(5, 3, 7, 9)),
    "evalmod_doubling_minus_one_dropped": (_doubling_without_minus_one,
                                           lambda bc: TB.test_evalmod_series_and_doublings()),
    "stage_groups_out_of_order": (_stage_groups_reversed, lambda bc: TB.test_stage_groups_cover_every_stage()),
    "crt_lift_not_centred": (_crt_not_centred, lambda bc: S.test_encrypt_decrypt_noise_bound(_tiny())),
    "galois_generator_3": (_galois_generator_3, lambda bc: S.test_rotate_moves_slots()),
    "repack_shift_reversed": (_repack_shift_reversed,
                              lambda bc: TL.test_repack_moves_every_value((16, 2, 256), (8, 1, 64))),
    "mod_raise_uncentred": (_raise_uncentred, lambda bc: TB.test_mod_raise_is_exact(bc)),
    "pool_mask_one_over_k": (_pool_mask_one_over_k,
                             lambda bc: TL.test_avgpool_plan_is_average_pooling(2, 2, 2, 8, 8, 1)),
    "fold_rotation_sign": (_fold_rotated_the_wrong_way,
                           lambda bc: TL.test_fc_diag_plan_is_the_product(16, 4, 28, 4, 12)),
    "conjugation_monomial_sign": (_monomial_sign, lambda bc: TB.test_bootstrap_encrypted(bc)),
    # the sparse bootstrap
    "sparse_copy_factor_conjugated": (_copy_factor_conjugated,
                                      lambda bc: TB.test_sparse_transforms_on_the_subring(64, 16)),
    "sparse_join_map_swapped": (_join_map_swapped, lambda bc: TB.test_sparse_transforms_on_the_subring(64, 32)),
    "sparse_trace_skipped": (_trace_skipped, lambda bc: TB.test_sparse_bootstrap_encrypted(bc)),
    # the paper's own layer algorithms (Sec. 5.1, 5.2, 5.4, 5.5)
    "paper_pad_row_gap_P": (_rotation_remapped(lambda r: -1 if r == -2 else r),
                            lambda bc: TP.test_padding_by_rotations(3, 5, 5, 1)),
    "paper_channel_sum_by_W": (_rotation_remapped(lambda r: 6 if r == 36 else r),
                               lambda bc: TP.test_conv_is_the_convolution_with_k_plus_f_keys(2, 3, 3, 6, 6)),
    "paper_extraction_one_too_far": (_rotation_remapped(lambda r: 3 if r == 2 else r),
                                     lambda bc: TP.test_conv_is_the_convolution_with_k_plus_f_keys(1, 1, 3, 6, 6)),
    "paper_stride_compaction_by_S": (_rotation_remapped(lambda r: 2 * r if r in (1, 2) else r),
                                     lambda bc: TP.test_striding_key_and_rotation_counts(8, 3, 2)),
    "paper_fc_merge_sign": (_rotation_remapped(lambda r: -r if -5 < r < 0 else r),
                            lambda bc: TP.test_fc_with_merge_budget(5, None)),
    "paper_global_pool_merge_by_block": (_rotation_remapped(lambda r: 64 if r == 63 else r),
                                         lambda bc: TP.test_global_avgpool(3, 8)),
}


@pytest.mark.parametrize("name", sorted(PY_PLANTS))
def test_planted_python_mistake_fails_its_pin(name, monkeypatch, request):
    plant, pin = PY_PLANTS[name]
    bc = (request.getfixturevalue("boot_ctx")
          if name in ("mod_raise_uncentred", "conjugation_monomial_sign", "sparse_trace_skipped") else None)
    plant(monkeypatch)
    with pytest.raises(AssertionError):
        pin(bc)
