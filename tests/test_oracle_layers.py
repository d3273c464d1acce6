"""Pins of the oracle's packed network layers: the rotation-sum plans of
convolution and average pooling and the FC plan, simulated exactly on FP64 slot
vectors, against the plain FP64 layers (Sec. 5.1, 4.4, 4.5 equations), also
chained on dilated grids; and the encrypted plans against the slot model under
decryption."""
import numpy as np
import pytest

from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth


@pytest.mark.parametrize("C,F,k,pad,H,grid,dil", [
    (1, 3, 3, 0, 6, 8, 1), (2, 3, 3, 1, 6, 8, 1), (3, 2, 5, 2, 5, 7, 1), (2, 2, 3, 0, 4, 10, 2)])
def test_conv_plan_is_the_convolution(C, F, k, pad, H, grid, dil):
    W = H
    block = max(dil * H * grid, 64)
    nslots = 1 << int(np.ceil(np.log2(max(C, F) * block + 1)))
    X = synth.image(11, C, (C, H, W), dist="normal")
    K = synth.conv_kernel(11, F, (F, C, k, k))
    want = OF.conv2d_fp64(X, K, pad=pad)
    rest = np.ones(nslots, bool)
    rest[OF.map_slots(*want.shape, grid, dil, block)] = False
    # every split of the block shifts into baby and giant steps is the same map
    for baby in (None, 1, 2, 3, C + F - 1):
        r, groups = OF.conv_plan(C, F, k, pad, H, W, grid, dil, block, nslots, K, baby=baby)
        y = OF.linear_slots(OF.pack_map(X, nslots, grid, dil, block), r, groups)
        assert np.max(np.abs(OF.unpack_map(y, want.shape, grid, dil, block) - want)) < 1e-12
        # nothing outside the output map
        assert np.max(np.abs(y[rest])) < 1e-12
        B = OF.conv_baby(k, C, F) if baby is None else baby
        assert len(r) == B * k * k and len(groups) <= -(-(C + F - 1) // B) + 1


def test_conv_baby_is_the_fewest_rotations():
    """B minimises B k^2 - 1 + 2 ceil((C + F - 1)/B), found by brute force."""
    for k in (1, 3, 5):
        for C, F in ((1, 6), (6, 16), (16, 16), (16, 32), (64, 64), (3, 4)):
            G = C + F - 1
            costs = [k * k * B - 1 + 2 * (-(-G // B)) for B in range(1, G + 1)]
            assert OF.conv_baby(k, C, F) == 1 + int(np.argmin(costs))


@pytest.mark.parametrize("C,F,k,pad,stride,H,grid,dil", [
    (2, 3, 3, 1, 2, 8, 8, 1), (1, 2, 3, 0, 2, 9, 10, 1), (2, 2, 3, 1, 2, 6, 14, 2)])
def test_strided_conv_plan(C, F, k, pad, stride, H, grid, dil):
    block = dil * H * grid
    nslots = 1 << int(np.ceil(np.log2(max(C, F) * block + 1)))
    X = synth.image(16, C, (C, H, H), dist="normal")
    K = synth.conv_kernel(16, F, (F, C, k, k))
    r, groups = OF.conv_plan(C, F, k, pad, H, H, grid, dil, block, nslots, K, stride=stride)
    y = OF.linear_slots(OF.pack_map(X, nslots, grid, dil, block), r, groups)
    want = OF.conv2d_fp64(X, K, stride=stride, pad=pad)
    assert np.max(np.abs(OF.unpack_map(y, want.shape, grid, dil * stride, block) - want)) < 1e-12


@pytest.mark.parametrize("C,k,stride,H,grid,dil", [(2, 2, 2, 8, 8, 1), (3, 2, 2, 4, 12, 2), (1, 3, 1, 5, 6, 1)])
def test_avgpool_plan_is_average_pooling(C, k, stride, H, grid, dil):
    block = dil * H * grid
    nslots = 1 << int(np.ceil(np.log2(C * block + 1)))
    X = synth.image(12, C, (C, H, H))
    r, groups = OF.avgpool_plan(C, k, stride, H, H, grid, dil, block, nslots)
    y = OF.linear_slots(OF.pack_map(X, nslots, grid, dil, block), r, groups)
    want = OF.avgpool_fp64(X, k, stride)
    assert np.max(np.abs(OF.unpack_map(y, want.shape, grid, dil * stride, block) - want)) < 1e-12


def test_fc_plan_is_the_product():
    nslots = 256
    slots = np.array([3, 7, 20, 21, 40, 100, 101, 200])
    Wm = synth.image(13, 0, (5, len(slots)), dist="normal")
    x = synth.image(13, 1, (len(slots),), dist="normal")
    v = np.zeros(nslots)
    v[slots] = x
    ws, es = OF.fc_plan(Wm, slots, nslots)
    y = OF.fc_slots(v, ws, es)
    assert np.max(np.abs(y[:5] - Wm @ x)) < 1e-12 and np.max(np.abs(y[5:])) == 0.0
    # the rotate-and-add steps leave the total in every slot
    t = v.copy()
    for s in OF.slot_sum_steps(nslots):
        t = t + np.roll(t, -s)
    assert np.max(np.abs(t - v.sum())) < 1e-12


@pytest.mark.parametrize("C,H,grid,dil,m", [(16, 4, 28, 4, 12), (3, 5, 12, 2, 7), (1, 10, 10, 1, 5), (5, 3, 8, 2, 4)])
def test_fc_diag_plan_is_the_product(C, H, grid, dil, m):
    block = dil * H * grid
    nslots = 1 << int(np.ceil(np.log2(C * block + 1)))
    X = synth.image(17, C, (C, H, H), dist="normal")
    Wm = synth.image(17, 99, (m, C * H * H), dist="normal")
    v = OF.pack_map(X, nslots, grid, dil, block)
    fold, r, groups = OF.fc_diag_plan(Wm, C, H, H, grid, dil, block, nslots)
    y = OF.linear_slots(OF.fold_slots(v, fold), r, groups)
    assert np.max(np.abs(y[:m] - Wm @ X.reshape(-1))) < 1e-12
    assert np.max(np.abs(y[m:])) < 1e-12
    # far fewer rotations than one slot sum per neuron
    assert len(OF.linear_steps(r, groups)) + len(fold) < m * int(np.log2(nslots))


def test_chained_layers_on_dilated_grids():
    """conv (valid) -> avgpool 2/2 -> conv on the stride-2 grid -> FC, as the
    slot model, against the FP64 chain."""
    grid, block, nslots = 12, 144, 1024
    X = synth.image(14, 0, (1, 12, 12))
    K1 = synth.conv_kernel(14, 1, (2, 1, 3, 3))
    K2 = synth.conv_kernel(14, 2, (3, 2, 3, 3))
    Wm = synth.image(14, 3, (4, 3 * 3 * 3), dist="normal")
    v = OF.pack_map(X, nslots, grid, 1, block)
    r, g = OF.conv_plan(1, 2, 3, 0, 12, 12, grid, 1, block, nslots, K1)
    v = OF.linear_slots(v, r, g)                                     # (2, 10, 10), dil 1
    r, g = OF.avgpool_plan(2, 2, 2, 10, 10, grid, 1, block, nslots)
    v = OF.linear_slots(v, r, g)                                     # (2, 5, 5), dil 2
    r, g = OF.conv_plan(2, 3, 3, 0, 5, 5, grid, 2, block, nslots, K2)
    v = OF.linear_slots(v, r, g)                                     # (3, 3, 3), dil 2
    ws, es = OF.fc_plan(Wm, OF.map_slots(3, 3, 3, grid, 2, block), nslots)
    y = OF.fc_slots(v, ws, es)
    h = OF.conv2d_fp64(OF.avgpool_fp64(OF.conv2d_fp64(X, K1), 2, 2), K2)
    assert np.max(np.abs(y[:4] - Wm @ h.reshape(-1))) < 1e-12


@pytest.fixture(scope="module")
def ctx11():
    P = synth.params("relu_n12")
    N = 1 << 11
    mods = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    L = len(P["qbits"])
    ctx = ckks.Ctx(N, mods[:L], mods[L:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    return ctx, P, se, ctx.keygen_pk(se)


def _plain(ctx, v, level):
    return ctx.plain_from_coeffs(ckks.encode(v, ctx.N, float(ctx.q[level - 1])), level)


def test_encrypted_linear_plans_match_the_slot_model(ctx11):
    ctx, P, se, pk = ctx11
    N, n, D = ctx.N, ctx.N // 2, P["scale"]
    grid, block = 8, 64
    X = synth.image(15, 0, (2, 6, 6))
    K = synth.conv_kernel(15, 1, (3, 2, 3, 3))
    v = OF.pack_map(X, n, grid, 1, block)
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(v, N, D), 4), 6)
    lv = 6
    r, groups = OF.conv_plan(2, 3, 3, 1, 6, 6, grid, 1, block, n, K)
    keys = {s: ctx.rotkey(se, ckks.galois_elt(s, N)) for s in OF.linear_steps(r, groups)}
    pts = [[_plain(ctx, p, lv) if p is not None else None for p in vals] for _, vals in groups]
    y = OF.linear_encrypted(ctx, ct, r, groups, pts, keys)
    assert y.shape[1] == lv - 1
    got = ctx.decode_ct(se, y, D).real
    assert np.max(np.abs(got - OF.linear_slots(v, r, groups))) < 1e-5
    # FC on that output
    slots = OF.map_slots(3, 6, 6, grid, 1, block)
    Wm = synth.image(15, 2, (4, len(slots)), dist="normal") * 0.1
    ws, es = OF.fc_plan(Wm, slots, n)
    lv2 = lv - 1
    keys.update({s: ctx.rotkey(se, ckks.galois_elt(s, N)) for s in OF.slot_sum_steps(n) if s not in keys})
    z = OF.fc_encrypted(ctx, y, [_plain(ctx, w, lv2) for w in ws], [_plain(ctx, e, lv2 - 1) for e in es], keys)
    assert z.shape[1] == lv2 - 2
    got = ctx.decode_ct(se, z, D).real
    want = OF.fc_slots(OF.linear_slots(v, r, groups), ws, es)
    assert np.max(np.abs(got - want)) < 1e-4


def test_encrypted_fc_diag_matches_the_product(ctx11):
    ctx, P, se, pk = ctx11
    N, n, D = ctx.N, ctx.N // 2, P["scale"]
    C, H, grid, dil, block, m = 4, 3, 8, 2, 64, 6
    X = synth.image(18, 0, (C, H, H))
    Wm = synth.image(18, 1, (m, C * H * H), dist="normal") * 0.2
    v = OF.pack_map(X, n, grid, dil, block)
    lv = 5
    ct = ctx.drop_level(ctx.encrypt(pk, ckks.encode(v, N, D), 5), lv)
    fold, r, groups = OF.fc_diag_plan(Wm, C, H, H, grid, dil, block, n)
    assert fold
    steps = sorted(set(OF.linear_steps(r, groups)) | {f for f in fold if f})
    keys = {s: ctx.rotkey(se, ckks.galois_elt(s, N)) for s in steps}
    pts = [[_plain(ctx, p, lv) if p is not None else None for p in vals] for _, vals in groups]
    y = OF.linear_encrypted(ctx, OF.fold_encrypted(ctx, ct, fold, keys), r, groups, pts, keys)
    assert y.shape[1] == lv - 1
    got = ctx.decode_ct(se, y, D).real
    assert np.max(np.abs(got[:m] - Wm @ X.reshape(-1))) < 1e-4
    assert np.max(np.abs(got[m:])) < 1e-4


@pytest.mark.parametrize("src,dst", [((16, 2, 256), (8, 1, 64)), ((16, 2, 256), (8, 1, 256)), ((8, 1, 256), (8, 1, 64))])
def test_repack_moves_every_value(src, dst):
    """Repacking by masks and rotations: every (c, i, j) lands at its slot in
    the new layout (brute-force pack/unpack), every other slot is zero."""
    n, shape = 2048, (8, 8, 8)
    X = synth.image(0xAB01, 0, shape, dist="normal")
    r, groups = OF.repack_plan(*shape, src, dst, n)
    out = OF.plan_slots(OF.pack_map(X, n, *src), r, groups).real
    assert np.array_equal(OF.unpack_map(out, shape, *dst), X)
    mask = np.ones(n, dtype=bool)
    mask[OF.map_slots(*shape, *dst)] = False
    assert np.all(out[mask] == 0.0)


@pytest.mark.parametrize("baby", [None, 2, 3])
def test_conv_plan_with_shared_tap_steps(baby):
    """A dilated map whose taps span more than a block (8 channels of 2x2 on
    a 4-wide grid, dilation 2, blocks of 16 slots): baby steps r - a*block of
    different taps coincide and are merged; the plan is still the convolution."""
    C, F, k, pad, H, grid, dil, block = 8, 8, 3, 1, 2, 4, 2, 16
    nslots = 256
    X = synth.image(18, C, (C, H, H), dist="normal")
    K = synth.conv_kernel(18, F, (F, C, k, k))
    r, groups = OF.conv_plan(C, F, k, pad, H, H, grid, dil, block, nslots, K, baby=baby)
    B = OF.conv_baby(k, C, F) if baby is None else baby
    assert B > 1 and len(set(r)) == len(r) < B * k * k
    y = OF.linear_slots(OF.pack_map(X, nslots, grid, dil, block), r, groups)
    want = OF.conv2d_fp64(X, K, pad=pad)
    assert np.max(np.abs(OF.unpack_map(y, want.shape, grid, dil, block) - want)) < 1e-12
