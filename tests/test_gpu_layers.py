"""Packed network layers on the GPU: the rotation-sum plans (multi-channel
conv with block shifts, average pooling on a dilated grid) and the FC plan
against the oracle's encrypted plans from the same integer plaintexts,
bit-exact; the layers built from weights on the device against the FP64
layers; key and map queries."""
import numpy as np
import pytest

import gpu_common
from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

GRID, BLOCK = 8, 64


@pytest.fixture(scope="module")
def pair():
    return gpu_common.Pair("relu_n12")


def _enc_map(pr, X, dil, nonce, level):
    v = OF.pack_map(X, pr.N // 2, GRID, dil, BLOCK)
    ct, oct_ = pr.encrypt_both(ckks.encode(v, pr.N, pr.P["scale"]), nonce=nonce, level=level)
    return v, ct, oct_


def _plains(pr, vals, level, scale):
    """The same integer plaintext on both sides (None stays None)."""
    g, o = [], []
    for v in vals:
        if v is None:
            g.append(None)
            o.append(None)
            continue
        m = ckks.encode(v, pr.N, scale)
        g.append(pr.g.plain_from_coeffs(m, pr.L, scale))
        o.append(pr.o.plain_from_coeffs(m, pr.L))
    return g, o


def _linear_pair(pr, r, groups, level):
    scale = float(pr.g.moduli[level - 1])
    gp, op = [], []
    for _, vals in groups:
        a, b = _plains(pr, vals, level, scale)
        gp.append(a)
        op.append(b)
    pr.add_keys(OF.linear_steps(r, groups))
    okeys = {s: pr.okeys[pr.g.galois_elt(s)] for s in OF.linear_steps(r, groups)}
    layer = pr.g.linear_prepare_plain(r, [s for s, _ in groups], gp, level)
    return layer, op, okeys, gp


def test_conv_plan_bit_exact(pair):
    X = synth.image(80, 0, (2, 6, 6))
    K = synth.conv_kernel(80, 1, (3, 2, 3, 3))
    level = 6
    v, ct, oct_ = _enc_map(pair, X, 1, 8000, level)
    r, groups = OF.conv_plan(2, 3, 3, 1, 6, 6, GRID, 1, BLOCK, pair.N // 2, K)
    layer, op, okeys, keep = _linear_pair(pair, r, groups, level)
    y = pair.g.layer_apply(layer, ct)
    want = OF.linear_encrypted(pair.o, oct_, r, groups, op, okeys)
    assert gpu_common.mismatch(pair.g.ct_download(y), want) == 0
    assert sorted(pair.g.layer_rotation_steps(layer)) == OF.linear_steps(r, groups)


def test_avgpool_plan_bit_exact(pair):
    X = synth.image(81, 0, (3, 4, 4))
    level = 5
    v, ct, oct_ = _enc_map(pair, X, 2, 8100, level)
    r, groups = OF.avgpool_plan(3, 2, 2, 4, 4, GRID, 2, BLOCK, pair.N // 2)
    layer, op, okeys, keep = _linear_pair(pair, r, groups, level)
    y = pair.g.layer_apply(layer, ct)
    want = OF.linear_encrypted(pair.o, oct_, r, groups, op, okeys)
    assert gpu_common.mismatch(pair.g.ct_download(y), want) == 0


def test_fc_plan_bit_exact(pair):
    X = synth.image(82, 0, (2, 3, 3))
    level = 5
    v, ct, oct_ = _enc_map(pair, X, 1, 8200, level)
    slots = OF.map_slots(2, 3, 3, GRID, 1, BLOCK)
    Wm = synth.image(82, 1, (4, len(slots)), dist="normal") * 0.2
    ws, es = OF.fc_plan(Wm, slots, pair.N // 2)
    gw, ow = _plains(pair, ws, level, float(pair.g.moduli[level - 1]))
    ge, oe = _plains(pair, es, level - 1, float(pair.g.moduli[level - 2]))
    steps = OF.slot_sum_steps(pair.N // 2)
    pair.add_keys(steps)
    layer = pair.g.fc_prepare_plain(gw, ge, level)
    y = pair.g.layer_apply(layer, ct)
    want = OF.fc_encrypted(pair.o, oct_, ow, oe, {s: pair.okeys[pair.g.galois_elt(s)] for s in steps})
    assert gpu_common.mismatch(pair.g.ct_download(y), want) == 0
    assert pair.g.layer_rotation_steps(layer) == steps


def test_strided_conv_bit_exact_and_from_weights(pair):
    X = synth.image(84, 0, (2, 7, 7))
    K = synth.conv_kernel(84, 1, (3, 2, 3, 3), std=0.3)
    level = 6
    v, ct, oct_ = _enc_map(pair, X, 1, 8400, level)
    r, groups = OF.conv_plan(2, 3, 3, 1, 7, 7, GRID, 1, BLOCK, pair.N // 2, K, stride=2)
    layer, op, okeys, keep = _linear_pair(pair, r, groups, level)
    y = pair.g.layer_apply(layer, ct)
    want = OF.linear_encrypted(pair.o, oct_, r, groups, op, okeys)
    assert gpu_common.mismatch(pair.g.ct_download(y), want) == 0
    # built from the weights on the device
    L = pair.g.conv_prepare((2, 7, 7, GRID, 1, BLOCK), K, 1, level, pair.P["scale"], stride=2)
    assert pair.g.layer_out_map(L) == (3, 4, 4, GRID, 2, BLOCK)
    pair.add_keys(pair.g.layer_rotation_steps(L))
    got = np.asarray(pair.g.decode(pair.g.decrypt(pair.sk, pair.g.layer_apply(L, ct)))).real
    want = OF.conv2d_fp64(X, K, stride=2, pad=1)
    assert np.max(np.abs(OF.unpack_map(got, want.shape, GRID, 2, BLOCK) - want)) < 1e-4


def test_fc_diag_bit_exact(pair):
    """The diagonal FC with the channel fold (4 channels on the dilation-2 grid)."""
    C, H, dil, m = 4, 3, 2, 6
    X = synth.image(85, 0, (C, H, H))
    Wm = synth.image(85, 1, (m, C * H * H), dist="normal") * 0.2
    level = 5
    v, ct, oct_ = _enc_map(pair, X, dil, 8500, level)
    fold, r, groups = OF.fc_diag_plan(Wm, C, H, H, GRID, dil, BLOCK, pair.N // 2)
    pair.add_keys([f for f in fold if f])
    layer, op, okeys, keep = _linear_pair(pair, r, groups, level)
    okeys.update({f: pair.okeys[pair.g.galois_elt(f)] for f in fold if f})
    layer = pair.g.linear_prepare_plain(r, [s for s, _ in groups], keep, level, fold=fold)
    y = pair.g.layer_apply(layer, ct)
    want = OF.linear_encrypted(pair.o, OF.fold_encrypted(pair.o, oct_, fold, okeys), r, groups, op, okeys)
    assert gpu_common.mismatch(pair.g.ct_download(y), want) == 0
    # built from the weights on the device
    L = pair.g.fc_prepare((C, H, H, GRID, dil, BLOCK), Wm, level, pair.P["scale"])
    pair.add_keys(pair.g.layer_rotation_steps(L))
    got = np.asarray(pair.g.decode(pair.g.decrypt(pair.sk, pair.g.layer_apply(L, ct)))).real
    assert np.max(np.abs(got[:m] - Wm @ X.reshape(-1))) < 1e-4 and np.max(np.abs(got[m:])) < 1e-4


def test_layers_from_weights_match_fp64(pair):
    """conv (valid, 1 -> 2) -> avgpool 2/2 -> conv (2 -> 3) on the stride-2 grid
    -> FC, each built from its weights on the device, decrypted against the
    FP64 chain."""
    g = pair.g
    D = pair.P["scale"]
    n = pair.N // 2
    grid, block = 12, 144
    X = synth.image(83, 0, (1, 12, 12))
    K1 = synth.conv_kernel(83, 1, (2, 1, 3, 3), std=0.3)
    b1 = np.array([0.1, -0.2])
    K2 = synth.conv_kernel(83, 2, (3, 2, 3, 3), std=0.3)
    Wm = synth.image(83, 3, (4, 27), dist="normal") * 0.2
    bf = np.array([0.5, 0.0, -0.5, 1.0])
    v = OF.pack_map(X, n, grid, 1, block)
    ct, _ = pair.encrypt_both(ckks.encode(v, pair.N, D), nonce=8300)
    lv = pair.L
    m0 = (1, 12, 12, grid, 1, block)
    L1 = g.conv_prepare(m0, K1, 0, lv, D, bias=b1)
    m1 = g.layer_out_map(L1)
    assert m1 == (2, 10, 10, grid, 1, block)
    L2 = g.avgpool_prepare(m1, 2, 2, lv - 1)
    m2 = g.layer_out_map(L2)
    assert m2 == (2, 5, 5, grid, 2, block)
    L3 = g.conv_prepare(m2, K2, 0, lv - 2, D)
    m3 = g.layer_out_map(L3)
    L4 = g.fc_prepare(m3, Wm, lv - 3, D, bias=bf)
    for layer in (L1, L2, L3, L4):
        pair.add_keys(g.layer_rotation_steps(layer))
    y = ct
    for layer in (L1, L2, L3, L4):
        y = g.layer_apply(layer, y)
    assert g.ct_info(y)[0] == lv - 4
    got = np.asarray(g.decode(g.decrypt(pair.sk, y))).real
    h = OF.conv2d_fp64(OF.avgpool_fp64(OF.conv2d_fp64(X, K1, b=b1), 2, 2), K2)
    want = Wm @ h.reshape(-1) + bf
    assert np.max(np.abs(got[:4] - want)) < 1e-3
    assert np.max(np.abs(got[4:])) < 1e-3


def test_one_shot_layers_and_key_budget(pair):
    """fheon_global_avgpool against the FP64 mean; fheon_fc within a key budget
    that admits its diagonal form and one that forces the paper's slot-sum
    form, both against the product; fheon_bootstrap on a context too shallow
    for it reports the level error."""
    g, D = pair.g, pair.P["scale"]
    C, H = 3, 4
    X = synth.image(86, 0, (C, H, H))
    m_in = (C, H, H, GRID, 1, BLOCK)
    v = OF.pack_map(X, pair.N // 2, GRID, 1, BLOCK)
    ct, _ = pair.encrypt_both(ckks.encode(v, pair.N, D), nonce=8600, level=6)
    lg = g.global_avgpool_prepare(m_in, 6)
    pair.add_keys(g.layer_rotation_steps(lg))
    got = np.asarray(g.decode(g.decrypt(pair.sk, g.global_avgpool(ct, m_in)))).real
    for c in range(C):
        assert abs(got[c * BLOCK] - X[c].mean()) < 1e-5
    Wm = synth.image(86, 1, (5, C * H * H), dist="normal") * 0.2
    want = Wm @ X.reshape(-1)
    steps = OF.slot_sum_steps(pair.N // 2)
    pair.add_keys(steps)
    L = g.fc_prepare(m_in, Wm, 6, D)
    pair.add_keys(g.layer_rotation_steps(L))
    for budget in (0, len(steps)):
        y = g.fc(ct, m_in, Wm, max_keys=budget)
        assert g.ct_info(y)[0] == (5 if budget == 0 else 4)
        got = np.asarray(g.decode(g.decrypt(pair.sk, y))).real
        assert np.max(np.abs(got[:5] - want)) < 1e-4
    with pytest.raises(pair.F.FheonError) as e:
        g.fc(ct, m_in, Wm, max_keys=3)
    assert e.value.code == -1
    with pytest.raises(pair.F.FheonError) as e:
        g.bootstrap(ct)
    assert e.value.code == -4


@pytest.mark.parametrize("C,F,k,s,p,H,levels", [(3, 4, 3, 2, 1, 8, 2), (1, 6, 5, 1, 0, 12, 2), (2, 3, 3, 1, 1, 8, 1)])
def test_conv2d_one_shot_general(pair, C, F, k, s, p, H, levels):
    """fheon_conv2d(in_ch, out_ch, k, stride, pad) on the flattened (C, H, W)
    map (Sec. 5.1-5.2): the compact (F, Ho, Wo) output within 1e-4 of the FP64
    convolution (decryption noise at scale 2^40 is ~1e-7), zero elsewhere; and
    the same ciphertext, bit for bit, as the two prepared layers it is made of
    (the rotation-sum conv, then the repack to the compact map when needed)."""
    pr = pair
    g = pr.g
    level = 8
    X = synth.image(95, C, (C, H, H))
    K = synth.conv_kernel(95, F, (F, C, k, k), std=0.3)
    b = synth.image(95, 99, (F,), dist="normal") * 0.1
    n = pr.N // 2
    x = np.zeros(n)
    x[:X.size] = X.reshape(-1)
    pr.add_keys(g.conv2d_rotation_steps(C, F, k, s, p, H, H))
    ct = g.drop_level(g.encrypt(pr.pk, g.encode(x, pr.L, pr.P["scale"]), nonce=9500 + C), level)
    out = g.conv2d(ct, C, F, k, s, p, H, H, K, bias=b)
    assert g.ct_info(out)[0] == level - levels
    want = OF.conv2d_fp64(X, K, b=b, stride=s, pad=p)
    y = np.asarray(g.decode(g.decrypt(pr.sk, out))).real
    assert np.max(np.abs(y[:want.size] - want.reshape(-1))) < 1e-4
    assert np.max(np.abs(y[want.size:])) < 1e-4
    # the composition of prepared layers
    conv = g.conv_prepare((C, H, H, H, 1, H * H), K, p, level, pr.P["scale"], bias=b, stride=s)
    mid = g.layer_apply(conv, ct)
    Ho = (H + 2 * p - k) // s + 1
    if levels == 2:
        rp = g.repack_prepare(g.layer_out_map(conv), (F, Ho, Ho, Ho, 1, Ho * Ho), level - 1)
        mid = g.layer_apply(rp, mid)
    assert gpu_common.mismatch(g.ct_download(out), g.ct_download(mid)) == 0


def test_conv2d_refuses_what_it_cannot_compute(pair):
    """A kernel larger than the padded input is refused by the key list and
    by the call, before any device work."""
    g = pair.g
    with pytest.raises(pair.F.FheonError) as e:
        g.conv2d_rotation_steps(1, 1, 9, 1, 0, 4, 4)
    assert e.value.code == -1
    ct = g.encrypt(pair.pk, g.encode(np.zeros(16), pair.L, pair.P["scale"]), nonce=9600)
    with pytest.raises(pair.F.FheonError) as e:
        g.conv2d(ct, 1, 2, 9, 1, 0, 4, 4, np.zeros((2, 1, 9, 9)))
    assert e.value.code == -1
