"""Pins of the bootstrapping oracle against what the mathematics fixes:
the butterfly factorisation of the slot transform against brute-force
evaluation at the slot roots and against the oracle's decode; merged levels
and their BSGS form against the stage-by-stage product; CoeffToSlot after
SlotToCoeff is the identity; the cosine series and its double-angle steps
against sin(2 pi y); ModRaise against exact integer arithmetic; and the whole
encrypted bootstrap against its input message and each intermediate against
the exact raised plaintext."""
import math

import numpy as np
import pytest

from oracle import boot as B
from oracle import ckks
from paper_2510_03996_gb300 import synth


def direct_slots(zp, N):
    """sum_k zp_k zeta_j^k at zeta_j = exp(i pi 5^j / N), j < N/2 (brute force)."""
    n = N // 2
    out = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e = pow(5, j, 2 * N)
        out[j] = sum(zp[k] * np.exp(1j * math.pi * ((e * k) % (2 * N)) / N) for k in range(n))
    return out


def brv_order(v):
    bits = len(v).bit_length() - 1
    return np.array([v[B.brv(j, bits)] for j in range(len(v))])


@pytest.mark.parametrize("n", [4, 16, 128])
def test_stages_are_the_slot_transform(n):
    N = 2 * n
    rng = synth.rng(0xB001, n)
    zp = rng.normal(size=n) + 1j * rng.normal(size=n)
    A = brv_order(zp)
    for s in range(1, n.bit_length()):
        A = B.apply_diagonals(B.stage_diagonals(n, 1 << (s - 1)), A)
    want = direct_slots(zp, N)
    assert np.max(np.abs(A - want)) < 1e-12 * n
    # the real polynomial (t_lo, t_hi) decodes to the same slots: zeta_j^(N/2) = i
    dec = ckks.decode(np.concatenate([zp.real, zp.imag]), n, 1.0)
    assert np.max(np.abs(dec - want)) < 1e-12 * n
    # inverse stages undo the stages one by one
    for s in range(1, n.bit_length()):
        S, Si = B.stage_diagonals(n, 1 << (s - 1)), B.stage_diagonals(n, 1 << (s - 1), inverse=True)
        v = rng.normal(size=n) + 1j * rng.normal(size=n)
        assert np.max(np.abs(B.apply_diagonals(Si, B.apply_diagonals(S, v)) - v)) < 1e-13


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_merged_levels_in_bsgs_form(levels):
    n = 256
    rng = synth.rng(0xB002, levels)
    zp = rng.normal(size=n) + 1j * rng.normal(size=n)
    v = brv_order(zp)
    seq = v.copy()
    for s in range(1, n.bit_length()):
        seq = B.apply_diagonals(B.stage_diagonals(n, 1 << (s - 1)), seq)
    x = v.copy()
    for stride, M in B.stc_levels(n, levels):
        r, groups = B.bsgs_plan(M, n, stride)
        assert r[0] == 0 and all(t % stride == 0 for t in r)
        x = B.plan_slots(x, r, groups)
    assert np.max(np.abs(x - seq)) < 1e-11
    for stride, M in B.cts_levels(n, levels):
        r, groups = B.bsgs_plan(M, n, stride)
        x = B.plan_slots(x, r, groups)
    assert np.max(np.abs(x - v)) < 1e-11
    # a fixed baby-step count gives the same map
    stride, M = B.stc_levels(n, levels)[0]
    r, groups = B.bsgs_plan(M, n, stride, baby=2)
    assert np.max(np.abs(B.plan_slots(v, r, groups) - B.apply_diagonals(M, v))) < 1e-11


def test_stage_groups_cover_every_stage():
    for logn in range(1, 16):
        for lv in range(1, logn + 1):
            g = B.stage_groups(logn, lv)
            assert [s for grp in g for s in grp] == list(range(1, logn + 1))
            assert max(map(len, g)) - min(map(len, g)) <= 1


def test_evalmod_series_and_doublings():
    for K in (128, 512):
        r = B.default_doublings(K)
        c = B.evalmod_coeffs(K, r)
        z = np.linspace(-1, 1, 2001)
        want = np.cos(2 * np.pi * (K * z - 0.25) / 2.0 ** r)
        assert np.max(np.abs(B.OF.cheb_eval_fp64(c, z) - want)) < 1e-13
        rng = synth.rng(0xB003, K)
        I = rng.integers(-K + 1, K, size=4000)
        eps = rng.uniform(-2 ** -8, 2 ** -8, size=I.size)
        got = B.evalmod_fp64((I + eps) / K, K, r)
        assert np.max(np.abs(got - np.sin(2 * np.pi * eps))) < 2e-9


def test_default_bound_and_depth():
    assert B.default_K(1 << 12) == 128 and B.default_K(1 << 16) == 512
    assert B.default_doublings(128) == 7 and B.default_doublings(512) == 9
    assert B.depth(3, 3, 27, 7) == 3 + B.OF.cheb_depth(27) + 7 + 3


@pytest.fixture(scope="module")
def boot_ctx():
    P = synth.params("boot_n12")
    N = 1 << P["logN"]
    L = len(P["qbits"])
    pr = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    ctx = ckks.Ctx(N, pr[:L], pr[L:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    plan = B.Plan(ctx, P["scale"])
    return P, ctx, s, se, pk, plan


def test_mod_raise_is_exact(boot_ctx):
    P, ctx, s, se, pk, plan = boot_ctx
    N = ctx.N
    z = synth.uniform_slots(0xB004, 0, N // 2)
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z, N, P["scale"]), 11), 1)
    q0 = int(ctx.q[0])
    low = ctx.decrypt_coeffs(se, ct)          # centred mod q_0
    raised = B.mod_raise(ctx, ct)
    assert raised.shape == (2, ctx.L, N)
    t = ctx.decrypt_coeffs(se, raised)        # exact integers over Q
    I = [(a - b) // q0 for a, b in zip(t, low)]
    assert all((a - b) % q0 == 0 for a, b in zip(t, low))
    assert max(abs(x) for x in I) < plan.K
    # every limb holds the centred lift of the level-1 coefficients
    c1 = ctx.to_coeff(np.ascontiguousarray(ct[1, :1]), 1)[0].astype(object)
    c1 = [int(v) - q0 if int(v) > q0 // 2 else int(v) for v in c1]
    r1 = ctx.to_coeff(raised[1], ctx.L)
    for i in (0, 5, ctx.L - 1):
        assert all(int(r1[i][k]) == c1[k] % int(ctx.q[i]) for k in range(0, N, 97))


def test_plan_levels_and_scales(boot_ctx):
    P, ctx, s, se, pk, plan = boot_ctx
    assert plan.out_level == ctx.L - B.depth(3, 3, plan.D, plan.r)
    assert abs(plan.out_scale / P["scale"] - 1) < 1e-12
    assert len(plan.cts) == 3 and len(plan.stc) == 3
    assert 0 not in plan.steps()


def test_bootstrap_encrypted(boot_ctx):
    P, ctx, s, se, pk, plan = boot_ctx
    N, n = ctx.N, ctx.N // 2
    keys = {st: ctx.rotkey(se, ckks.galois_elt(st, N)) for st in plan.steps()}
    ck = ctx.rotkey(se, 2 * N - 1)
    rlk = ctx.relinkey(se)
    pts = plan.encode(ctx)
    z = synth.uniform_slots(0xB005, 0, n)
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z, N, P["scale"]), 12), 2)
    tr = {}
    y, sc = B.bootstrap_encrypted(ctx, ct, plan, pts, keys, rlk, ck, trace=tr)
    assert y.shape == (2, plan.out_level, N) and sc == plan.out_scale
    out = ctx.decode_ct(se, y, sc)
    assert np.max(np.abs(out - z)) < 1e-4
    # CoeffToSlot: (t_lo + i t_hi) / (2 K q_0) in bit-reversed slot order
    q0 = float(ctx.q[0])
    t = np.array([float(v) for v in ctx.decrypt_coeffs(se, tr["raised"])])
    want = brv_order((t[:n] + 1j * t[n:]) / (2 * plan.K * q0))
    got = ctx.decode_ct(se, tr["cts"], plan.cts_scale)
    assert np.max(np.abs(got - want)) < 1e-10
    # EvalMod of each part: sin(2 pi t / q_0)
    for part, half in zip(tr["evalmod"], (t[:n], t[n:])):
        v = ctx.decode_ct(se, part, plan.evalmod_scale)
        assert np.max(np.abs(v.real - np.sin(2 * np.pi * brv_order(half) / q0))) < 1e-7
        assert np.max(np.abs(v.imag)) < 1e-7


def test_slot_transform_at_the_test_size():
    """At n = 2^11 (the N = 2^12 contexts): the butterfly stages equal the
    oracle's decode of the real polynomial (t_lo, t_hi), and the three merged
    levels of each transform in BSGS form (the split the bootstrap uses)
    round-trip."""
    n = 1 << 11
    rng = synth.rng(0xB006, 0)
    zp = rng.normal(size=n) + 1j * rng.normal(size=n)
    A = brv_order(zp)
    for s in range(1, n.bit_length()):
        A = B.apply_diagonals(B.stage_diagonals(n, 1 << (s - 1)), A)
    dec = ckks.decode(np.concatenate([zp.real, zp.imag]), n, 1.0)
    assert np.max(np.abs(A - dec)) < 1e-9
    x = brv_order(zp)
    for stride, M in B.stc_levels(n, 3):
        r, groups = B.bsgs_plan(M, n, stride)
        x = B.plan_slots(x, r, groups)
    assert np.max(np.abs(x - dec)) < 1e-9
    for stride, M in B.cts_levels(n, 3):
        r, groups = B.bsgs_plan(M, n, stride)
        x = B.plan_slots(x, r, groups)
    assert np.max(np.abs(x - brv_order(zp))) < 1e-11


# ---------------------------------------------------------------- sparse bootstrap
def subring_poly(T, copies):
    """The polynomial T(X^copies) of degree < copies * len(T)."""
    t = np.zeros(copies * len(T))
    t[::copies] = T
    return t


@pytest.mark.parametrize("n,ns", [(64, 32), (64, 16), (256, 32)])
def test_sparse_transforms_on_the_subring(n, ns):
    """For a real T with 2 ns coefficients, the N-ring polynomial T(X^(n/ns))
    has the slots of T in its own ring repeated in every copy (decode on
    both sides).  The sparse CoeffToSlot levels take those slots to
    u = brv(T_lo + i T_hi) in even copies and -i u in odd ones, so that
    y + conj(y) = 2 (brv T_lo, brv T_hi); the sparse SlotToCoeff levels take
    (brv T_lo, brv T_hi) back to the slots."""
    rng = synth.rng(0xB00C, n + ns)
    T = rng.normal(size=2 * ns)
    copies = n // ns
    slots = ckks.decode(subring_poly(T, copies), n, 1.0)
    own = ckks.decode(T, ns, 1.0)
    assert np.max(np.abs(slots - np.tile(own, copies))) < 1e-9
    x = slots
    for stride, M in B.cts_levels_sparse(n, ns, 3 if ns >= 8 else 1):
        r, groups = B.bsgs_plan(M, n, stride)
        x = B.plan_slots(x, r, groups)
    u = brv_order(T[:ns] + 1j * T[ns:])
    want = np.tile(np.concatenate([u, -1j * u]), n // (2 * ns))
    assert np.max(np.abs(x - want)) < 1e-9
    w = x + np.conj(x)
    assert np.max(np.abs(w - np.tile(2 * np.concatenate([brv_order(T[:ns]), brv_order(T[ns:])]), n // (2 * ns)))) < 1e-9
    v = np.tile(np.concatenate([brv_order(T[:ns]), brv_order(T[ns:])]), n // (2 * ns)).astype(np.complex128)
    for stride, M in B.stc_levels_sparse(n, ns, 3 if ns >= 8 else 1):
        r, groups = B.bsgs_plan(M, n, stride)
        v = B.plan_slots(v, r, groups)
    assert np.max(np.abs(v - slots)) < 1e-9


def test_sparse_plan_levels_keys_and_scales(boot_ctx):
    P, ctx, s, se, pk, plan = boot_ctx
    sp = B.Plan(ctx, P["scale"], slots=ctx.N // 4)
    assert sp.out_level == plan.out_level and abs(sp.out_scale / P["scale"] - 1) < 1e-12
    assert sp.trace_steps() == [ctx.N // 4]
    assert ctx.N // 4 in sp.steps() and 0 not in sp.steps()
    assert np.array_equal(sp.mask_slots(), np.concatenate([np.ones(ctx.N // 4), np.zeros(ctx.N // 4)]))


def test_sparse_bootstrap_encrypted(boot_ctx):
    """The encrypted sparse bootstrap: the input's slots [0, N/4) come back in
    both copies (whatever the other slots held); the traced plaintext is
    `copies` times an element of Z[X^copies] up to key-switching noise; the
    CoeffToSlot output is (u, -i u) with u = brv(T_lo + i T_hi) / (2 K q_0)
    for T the subring coefficients / copies; EvalMod's output is
    sin(2 pi (brv T_lo, brv T_hi) / q_0)."""
    P, ctx, s, se, pk, plan = boot_ctx
    N, n = ctx.N, ctx.N // 2
    sp = B.Plan(ctx, P["scale"], slots=N // 4)
    ns, copies = sp.ns, sp.copies
    keys = {st: ctx.rotkey(se, ckks.galois_elt(st, N)) for st in sp.steps()}
    pts = sp.encode(ctx)
    z = synth.uniform_slots(0xB00D, 0, n)
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z, N, P["scale"]), 13), 3)
    tr = {}
    y, sc = B.bootstrap_encrypted(ctx, ct, sp, pts, keys, ctx.relinkey(se), ctx.rotkey(se, 2 * N - 1), trace=tr,
                                  mask=sp.encode_mask(ctx))
    assert y.shape == (2, sp.out_level, N) and sc == sp.out_scale
    out = ctx.decode_ct(se, y, sc)
    assert np.max(np.abs(out - np.tile(z[:ns], 2))) < 1e-4
    # the repeated input: slots [0, ns) in both copies
    rep = ctx.decode_ct(se, tr["repeated"], P["scale"])
    assert np.max(np.abs(rep - np.tile(z[:ns], 2))) < 1e-6
    q0 = float(ctx.q[0])
    t = np.array([float(v) for v in ctx.decrypt_coeffs(se, tr["traced"])])
    off = np.delete(t, np.arange(0, N, copies))
    assert np.max(np.abs(off)) < 2.0 ** 20 < q0 / 2.0 ** 20
    T = t[::copies] / copies
    u = brv_order((T[:ns] + 1j * T[ns:]) / (2 * sp.K * q0))
    got = ctx.decode_ct(se, tr["cts"], sp.cts_scale)
    assert np.max(np.abs(got - np.concatenate([u, -1j * u]))) < 1e-10
    (part,) = tr["evalmod"]
    v = ctx.decode_ct(se, part, sp.evalmod_scale)
    want = np.sin(2 * np.pi * np.concatenate([brv_order(T[:ns]), brv_order(T[ns:])]) / q0)
    assert np.max(np.abs(v.real - want)) < 1e-7
    assert np.max(np.abs(v.imag)) < 1e-7


def test_sparse_unmasked_bootstrap_encrypted(boot_ctx):
    """An unmasked sparse plan on an input that is zero outside slots
    [0, N/4), at level 1 (no level for a mask): those slots come back in
    both copies."""
    P, ctx, s, se, pk, plan = boot_ctx
    N, n = ctx.N, ctx.N // 2
    sp = B.Plan(ctx, P["scale"], slots=N // 4, masked=False)
    assert not sp.masked and sp.steps() == B.Plan(ctx, P["scale"], slots=N // 4).steps()
    keys = {st: ctx.rotkey(se, ckks.galois_elt(st, N)) for st in sp.steps()}
    z = synth.uniform_slots(0xB00E, 0, n)
    z[N // 4:] = 0.0
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(z, N, P["scale"]), 14), 1)
    y, sc = B.bootstrap_encrypted(ctx, ct, sp, sp.encode(ctx), keys, ctx.relinkey(se), ctx.rotkey(se, 2 * N - 1))
    out = ctx.decode_ct(se, y, sc)
    assert np.max(np.abs(out - np.tile(z[:N // 4], 2))) < 1e-4
