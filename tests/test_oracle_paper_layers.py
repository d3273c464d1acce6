"""Pins of the paper's own layer algorithms (oracle/paper_layers.py): each
against the plain FP64 layer equations (Sec. 5.1 convolution, Sec. 5.2 output
sizes, Sec. 5.4 pooling, Sec. 5.5 FC), and against the paper's counts of
keys and rotations: K + F keys for a convolution (Sec. 5.1), W rotations per
channel and at most C + 3 keys for padding, at most W_out + 2 keys for
striding approach 1, log2(W_out) + 1 keys and about log2(W_out) + W_out
rotations for approach 2 (Sec. 5.2).  Then the library's rotation-sum plans
(block shifts, striding left in place, diagonal FC) against the paper's forms
on the same maps: the same values.  A planted wrong rotation amount fails a
pin."""
import math

import numpy as np
import pytest

from oracle import fheon as OF
from oracle import paper_layers as PL
from paper_2510_03996_gb300 import synth


def nslots_for(*sizes):
    return 1 << int(math.ceil(math.log2(max(sizes) + 1)))


def run_conv(C, F, k, H, W, seed, **kw):
    P, S = kw.get("P", 0), kw.get("S", 1)
    Hp, Wp = H + 2 * P, W + 2 * P
    n = nslots_for(2 * max(C, F) * Hp * Wp)
    X = synth.image(seed, C, (C, H, W), dist="normal")
    K = synth.conv_kernel(seed, F, (F, C, k, k))
    b = synth.image(seed, 77, (F,), dist="normal")
    cnt = PL.Counter(n)
    y = PL.conv_advanced(cnt, PL.Ct(PL.flatten(X, n)), C, H, W, K, b, **kw) if (P or S > 1) else \
        PL.conv(cnt, PL.Ct(PL.flatten(X, n)), C, H, W, K, b)
    want = OF.conv2d_fp64(X, K, b=b, stride=S, pad=P)
    return cnt, y, want, (X, K, b, n)


@pytest.mark.parametrize("C,F,k,H,W", [(1, 1, 3, 6, 6), (2, 3, 3, 6, 6), (3, 2, 5, 8, 8), (2, 2, 3, 5, 7),
                                       (4, 1, 3, 4, 4)])
def test_conv_is_the_convolution_with_k_plus_f_keys(C, F, k, H, W):
    cnt, y, want, _ = run_conv(C, F, k, H, W, seed=31)
    got = PL.unflatten(y.v, want.shape)
    assert np.max(np.abs(got - want)) < 1e-12
    assert np.max(np.abs(y.v[want.size:])) < 1e-12
    Ho, Wo = H - k + 1, W - k + 1
    K_ = k * k - 1
    # Sec. 5.1: the k^2 - 1 tap keys, the W^2 channel key (C > 1), a placement
    # key per output channel f >= 1; the extraction reuses the tap key k - 1
    assert len(cnt.keys) == K_ + (1 if C > 1 else 0) + (F - 1)
    if C > 1:
        assert len(cnt.keys) == K_ + F
    assert (k - 1) in cnt.keys and {i * W + j for i in range(k) for j in range(k)} - {0} <= cnt.keys
    assert len(cnt.rotations) == K_ + F * (C - 1) + F * (Ho - 1) + (F - 1)
    # kernel products, the A* mask (C > 1), the row masks
    assert cnt.products == F * (k * k + (1 if C > 1 else 0) + Ho)
    assert y.depth == 2 + (1 if C > 1 else 0)


@pytest.mark.parametrize("C,H,W,P", [(1, 4, 4, 1), (3, 5, 5, 1), (2, 6, 4, 2), (4, 3, 3, 1)])
def test_padding_by_rotations(C, H, W, P):
    n = nslots_for(C * (H + 2 * P) * (W + 2 * P))
    X = synth.image(32, C, (C, H, W), dist="normal")
    cnt = PL.Counter(n)
    y = PL.pad(cnt, PL.Ct(PL.flatten(X, n)), C, H, W, P)
    want = np.pad(X, ((0, 0), (P, P), (P, P)))
    assert np.max(np.abs(PL.unflatten(y.v, want.shape) - want)) == 0.0
    assert np.max(np.abs(y.v[want.size:])) == 0.0
    # Sec. 5.2: H rotations per channel (W for a square map); C + 1 keys <= C + 3
    assert len(cnt.rotations) == C * H
    if H == W:
        assert len(cnt.rotations) == C * W
    assert len(cnt.keys) == C + 1 <= C + 3
    assert y.depth == 1


@pytest.mark.parametrize("C,F,k,H,P,S", [(2, 2, 3, 8, 1, 2), (1, 3, 3, 9, 0, 2), (3, 2, 3, 6, 1, 3),
                                         (2, 1, 5, 10, 2, 2), (1, 1, 3, 16, 1, 2)])
@pytest.mark.parametrize("approach,joint", [(1, False), (2, False), (2, True)])
def test_strided_padded_conv(C, F, k, H, P, S, approach, joint):
    cnt, y, want, _ = run_conv(C, F, k, H, H, seed=33, P=P, S=S, approach=approach, joint=joint)
    assert np.max(np.abs(PL.unflatten(y.v, want.shape) - want)) < 1e-12
    assert np.max(np.abs(y.v[want.size:])) < 1e-12


@pytest.mark.parametrize("Wa,Ho,S", [(8, 3, 2), (12, 5, 2), (10, 3, 3), (34, 16, 2)])
def test_striding_key_and_rotation_counts(Wa, Ho, S):
    """Striding alone on a stride-1 map A* (one channel at block 0)."""
    Wo = Ho
    n = nslots_for(2 * Wa * Wa)
    A = synth.image(34, 0, (Wa, Wa), dist="normal")
    v = PL.Ct(PL.flatten(A, n))
    want = A[0:S * Ho:S, 0:S * Wo:S]
    c1 = PL.Counter(n)
    y1 = PL.stride_extract(c1, v, Wa, Ho, Wo, S)
    assert np.max(np.abs(PL.unflatten(y1.v, (Ho, Wo)) - want)) == 0.0
    # approach 1: W_out + 1 keys (the paper: W_out + 2)
    assert len(c1.keys) == Wo + 1 <= Wo + 2
    c2 = PL.Counter(n)
    y2 = PL.stride_masks(c2, v, Wa, Wa * Wa, Ho, Wo, S)
    assert np.max(np.abs(PL.unflatten(y2.v, (Ho, Wo)) - want)) == 0.0
    lg = math.ceil(math.log2(Wo))
    # approach 2: log2(W_out) + 1 keys, log2(W_out) + W_out - 1 rotations
    assert len(c2.keys) == lg + 1
    assert len(c2.rotations) == lg + Ho - 1 <= lg + Wo
    assert c2.products == 1 + 2 * lg + Ho
    # approach 1 spends no level on the compaction but many rotations; approach 2 the reverse
    assert y1.depth == 1 < y2.depth == lg + 2
    assert len(c1.rotations) > len(c2.rotations)


@pytest.mark.parametrize("C,H,k,S", [(2, 8, 2, 2), (3, 6, 3, 3), (1, 9, 3, 2), (4, 4, 2, 2)])
@pytest.mark.parametrize("approach", [1, 2])
def test_avgpool(C, H, k, S, approach):
    n = nslots_for(2 * C * H * H)
    X = synth.image(35, C, (C, H, H))
    cnt = PL.Counter(n)
    y = PL.avgpool(cnt, PL.Ct(PL.flatten(X, n)), C, H, H, k, S, approach=approach)
    want = OF.avgpool_fp64(X, k, S)
    assert np.max(np.abs(PL.unflatten(y.v, want.shape) - want)) < 1e-14


@pytest.mark.parametrize("C,H", [(1, 4), (3, 8), (16, 2)])
def test_global_avgpool(C, H):
    n = nslots_for(2 * C * H * H)
    X = synth.image(36, C, (C, H, H), dist="normal")
    cnt = PL.Counter(n)
    y = PL.global_avgpool(cnt, PL.Ct(PL.flatten(X, n)), C, H, H)
    assert np.max(np.abs(y.v[:C] - X.mean(axis=(1, 2)))) < 1e-13
    assert np.max(np.abs(y.v[C:])) < 1e-13
    lg = int(math.log2(H * H))
    assert len(cnt.keys) == lg + (1 if C > 1 else 0)
    assert len(cnt.rotations) == lg + C - 1


@pytest.mark.parametrize("m,max_keys", [(5, None), (10, 9), (10, 3), (7, 1), (12, 4)])
def test_fc_with_merge_budget(m, max_keys):
    n = 256
    slots = np.array([0, 3, 7, 20, 21, 40, 100, 101, 200, 255])
    Wm = synth.image(37, 0, (m, len(slots)), dist="normal")
    x = synth.image(37, 1, (len(slots),), dist="normal")
    b = synth.image(37, 2, (m,), dist="normal")
    v = np.zeros(n)
    v[slots] = x
    cnt = PL.Counter(n)
    y = PL.fc(cnt, PL.Ct(v), Wm, b, slots, max_keys=max_keys)
    assert np.max(np.abs(y.v[:m] - (Wm @ x + b))) < 1e-12
    assert np.max(np.abs(y.v[m:])) < 1e-12
    sum_keys = {1 << t for t in range(int(math.log2(n)))}
    merge = cnt.keys - sum_keys
    if max_keys is None or max_keys >= m - 1:
        # Sec. 5.5: one merge key per output neuron (m - 1 of them)
        assert merge == {-kk for kk in range(1, m)}
    else:
        assert len(merge) <= max_keys
    assert y.depth == 2


# ------------------------------------------------------------------ the library's plans against the paper's forms
@pytest.mark.parametrize("C,F,k,H,P,S", [(1, 6, 5, 12, 0, 1), (2, 3, 3, 8, 1, 1), (2, 2, 3, 8, 1, 2),
                                         (3, 4, 3, 6, 1, 2)])
def test_block_shift_conv_gives_the_paper_conv(C, F, k, H, P, S):
    """The rotation-sum conv plan (one group per block shift, outputs left at
    stride-aligned slots) and the paper's pipeline (padding by rotations, A*,
    extraction or striding) give the same map on the same input."""
    cnt, y, want, (X, K, b, n) = run_conv(C, F, k, H, H, seed=38, P=P, S=S, approach=2)
    grid, block = H, H * H
    nsl = nslots_for(max(C, F) * block)
    r, groups = OF.conv_plan(C, F, k, P, H, H, grid, 1, block, nsl, K, stride=S)
    z = OF.linear_slots(OF.pack_map(X, nsl, grid, 1, block), r, groups)
    ours = OF.unpack_map(z, want.shape, grid, S, block) + b[:, None, None]
    paper = PL.unflatten(y.v, want.shape)
    assert np.max(np.abs(ours - paper)) < 1e-12


@pytest.mark.parametrize("C,H,k,S", [(6, 24, 2, 2), (16, 8, 2, 2)])
def test_in_place_pooling_gives_the_paper_pooling(C, H, k, S):
    n = nslots_for(2 * C * H * H)
    X = synth.image(39, C, (C, H, H))
    cnt = PL.Counter(n)
    y = PL.avgpool(cnt, PL.Ct(PL.flatten(X, n)), C, H, H, k, S)
    r, groups = OF.avgpool_plan(C, k, S, H, H, H, 1, H * H, n)
    z = OF.linear_slots(OF.pack_map(X, n, H, 1, H * H), r, groups)
    Ho = (H - k) // S + 1
    assert np.max(np.abs(OF.unpack_map(z, (C, Ho, Ho), H, S, H * H) - PL.unflatten(y.v, (C, Ho, Ho)))) < 1e-14


def test_diagonal_fc_gives_the_paper_fc():
    C, H, grid, dil, m = 3, 4, 16, 2, 10
    block = dil * H * grid
    n = nslots_for(C * block)
    X = synth.image(40, C, (C, H, H), dist="normal")
    Wm = synth.image(40, 9, (m, C * H * H), dist="normal")
    v = OF.pack_map(X, n, grid, dil, block)
    fold, r, groups = OF.fc_diag_plan(Wm, C, H, H, grid, dil, block, n)
    ours = OF.linear_slots(OF.fold_slots(v, fold), r, groups)[:m]
    cnt = PL.Counter(n)
    paper = PL.fc(cnt, PL.Ct(v), Wm, None, OF.map_slots(C, H, H, grid, dil, block))
    assert np.max(np.abs(ours - paper.v[:m])) < 1e-12


def plan_cost(r, groups, fold=()):
    """Rotations, keys and levels of a rotation-sum plan (taps hoisted)."""
    rots = [x for x in r if x] + [s for s, _ in groups if s] + [f for f in fold if f]
    return len(rots), len(set(rots)), 1


@pytest.mark.parametrize("name,C,F,k,H,P,S", [
    ("LeNet-5 conv 1", 1, 6, 5, 28, 0, 1), ("LeNet-5 conv 2", 6, 16, 5, 12, 0, 1),
    ("ResNet-20 stage-1 conv", 16, 16, 3, 32, 1, 1), ("ResNet-20 stage-2 first conv", 16, 32, 3, 32, 1, 2)])
def test_cost_of_the_block_shift_form(name, C, F, k, H, P, S):
    """The paper's convolution pipeline against the library's block-shift
    plan on the networks' layers (counted by the two planners): the plan uses
    one level instead of three or more, and fewer rotations."""
    Hp = H + 2 * P
    Ho = (Hp - k) // S + 1
    lg = math.ceil(math.log2(Ho))
    # the paper's form, counted from its steps (not run: the counts are closed forms pinned above)
    pad_rot = C * H if P else 0
    paper_rot = (k * k - 1) + F * (C - 1) + pad_rot + (F * (Ho - 1) if S == 1 else F * (lg + Ho - 1)) + (F - 1)
    paper_depth = (1 if P else 0) + 1 + (1 if C > 1 else 0) + (1 if S == 1 else lg + 2)
    block = H * H
    n = nslots_for(max(C, F) * block)
    K = np.ones((F, C, k, k))
    r, groups = OF.conv_plan(C, F, k, P, H, H, H, 1, block, n, K, stride=S)
    rot, keys, depth = plan_cost(r, groups)
    assert depth < paper_depth and rot < paper_rot, (name, rot, paper_rot)
