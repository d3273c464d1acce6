"""Pins of the oracle's FHEON layer packing: Algorithms 2-3 masks against tap
validity by brute force, the slot-level special convolution against the FP64
convolution equation, and the encrypted special conv against FP64."""
import numpy as np
import pytest

from oracle import ckks, fheon
from paper_2510_03996_gb300 import synth


def _conv_direct(X, K, pad):
    """Direct loops over the zero-padded input (a second, independent reading of
    the conv equation: out-of-range input reads as zero)."""
    C, H, W = X.shape
    F, _, k, _ = K.shape
    Y = np.zeros((F, H + 2 * pad - k + 1, W + 2 * pad - k + 1))
    for f in range(F):
        for h in range(Y.shape[1]):
            for w in range(Y.shape[2]):
                s = 0.0
                for c in range(C):
                    for i in range(k):
                        for j in range(k):
                            y, x = h + i - pad, w + j - pad
                            if 0 <= y < H and 0 <= x < W:
                                s += X[c, y, x] * K[f, c, i, j]
                Y[f, h, w] = s
    return Y


def test_conv2d_fp64_matches_direct_loops():
    X = synth.image(1, 0, (2, 7, 7))
    K = synth.conv_kernel(1, 1, (3, 2, 3, 3))
    for pad in (0, 1):
        assert np.allclose(fheon.conv2d_fp64(X, K, pad=pad), _conv_direct(X, K, pad))
    # stride: a subsample of the stride-1 output
    assert np.allclose(fheon.conv2d_fp64(X, K, stride=2, pad=1), fheon.conv2d_fp64(X, K, pad=1)[:, ::2, ::2])


@pytest.mark.parametrize("W,C", [(4, 1), (5, 2), (28, 1), (32, 3)])
def test_algorithm3_masks_are_tap_validity(W, C):
    masks = fheon.algorithm3_masks(W, C)
    for mask, (di, dj) in zip(masks, fheon.taps(3)):
        assert np.array_equal(mask, fheon.tap_mask(W, W, C, di, dj))


def test_build_mask_worked_case():
    # W = 3, tap (-1,-1): first row and first column invalid
    m = fheon.build_mask(3 + 1, 0, 3 - 1, 9, 1)
    assert list(m) == [0, 0, 0, 0, 1, 1, 0, 1, 1]


@pytest.mark.parametrize("k,C,H,W", [(3, 1, 6, 6), (3, 2, 5, 5), (5, 1, 28, 28), (5, 3, 7, 9)])
def test_special_conv_slots_equals_fp64_same_conv(k, C, H, W):
    n = 4096
    X = synth.image(2, k, (C, H, W))
    K = synth.conv_kernel(2, k, (1, C, k, k))
    x = np.zeros(n)
    x[:C * H * W] = X.reshape(-1)
    y = fheon.special_conv_slots(x, H, W, C, K[0], k)
    ref = fheon.conv2d_fp64(X, K, pad=(k - 1) // 2)
    assert np.allclose(y[:H * W], ref.reshape(-1), atol=1e-12)
    assert np.all(y[H * W:] == 0)


def test_rotation_step_count():
    # one key per non-identity tap: k^2 - 1 (paper Sec. 5.1: k^2 - 1 rotations)
    for k in (3, 5):
        steps = fheon.conv_rotation_steps(28, k)
        assert len(steps) == k * k - 1 and len(set(steps)) == k * k - 1 and 0 not in steps


@pytest.mark.parametrize("hoisted", [False, True])
def test_encrypted_special_conv_matches_fp64(hoisted):
    """Config-1 geometry (1x28x28, 5x5, pad 2) at N = 2^11 to keep the oracle fast;
    tap rotations one by one or hoisted."""
    P = synth.params("conv_n13")
    N = 1 << 11
    mods = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    ctx = ckks.Ctx(N, mods[:3], mods[3:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    pk = ctx.keygen_pk(se)
    H = W = 28
    k = 5
    X = synth.image(P["seed"], 0, (1, H, W))
    K = synth.conv_kernel(P["seed"], 1, (1, 1, k, k))
    x = np.zeros(N // 2)
    x[:H * W] = X.reshape(-1)
    ct = ctx.encrypt(pk, ckks.encode(x, N, P["scale"]), 0)
    keys = {r: ctx.rotkey(se, ckks.galois_elt(r, N)) for r in fheon.conv_rotation_steps(W, k)}
    taps = fheon.encode_tap_plains(ctx, H, W, K[0], k, 3)
    out = fheon.special_conv_encrypted(ctx, ct, keys, H, W, k, taps, hoisted=hoisted)
    assert out.shape[1] == 2
    y = ctx.decode_ct(se, out, P["scale"]).real
    ref = fheon.conv2d_fp64(X, K, pad=2).reshape(-1)
    assert np.max(np.abs(y[:H * W] - ref)) < 1e-4
    assert np.max(np.abs(y[H * W:])) < 1e-4
