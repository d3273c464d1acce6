"""Host side of the LeNet-5 runner: its FP64 forward pass (used to choose the
ReLU bounds) against the oracle's plain FP64 layers, the level budget, and
the layer chain on a stand-in context that passes every kernel and weight
matrix through the binding's own size checks."""
import numpy as np

from oracle import fheon as OF
from paper_2510_03996_gb300 import fheon as F
from paper_2510_03996_gb300 import lenet, synth


def test_fp64_forward_matches_the_oracle_layers():
    w = lenet.weights(synth.SEED_BASE + 2)
    for s in range(3):
        X = synth.image(90, s, (1, 28, 28))
        assert np.max(np.abs(lenet.forward_fp64(X, w) - OF.lenet_fp64(X, w))) < 1e-12


def test_level_budget_and_bounds():
    P = synth.params("lenet_n15")
    assert lenet.levels() == 7 + 4 * (OF.cheb_depth(59) + 1) and len(P["qbits"]) >= lenet.levels() + 2
    w = lenet.weights(synth.SEED_BASE + 2)
    xs = [synth.image(91, s, (1, 28, 28)) for s in range(4)]
    betas = lenet.relu_bounds(xs, w)
    assert len(betas) == 4 and all(b >= 1.0 for b in betas)
    # every ReLU input of the calibration set lies inside [-beta/1.5, beta/1.5]
    for X in xs:
        rec = []
        lenet.forward_fp64(X, w, record=rec)
        assert all(np.max(np.abs(r)) * 1.5 <= b + 1e-12 for r, b in zip(rec, betas))


class _ShapeCtx:
    """Maps and levels only; the weights go through the binding's checks."""

    def __init__(self):
        self.kinds = []

    def conv_prepare(self, m, K, pad, level, scale, bias=None, stride=1):
        F.Context._conv_weights(m, K, bias)
        C, H, W, grid, dil, block = m
        k = K.shape[2]
        self.kinds.append("conv")
        return (K.shape[0], (H + 2 * pad - k) // stride + 1, (W + 2 * pad - k) // stride + 1, grid, dil * stride, block)

    def relu_prepare(self, beta, degree, n, level):
        assert n >= 1 and level >= 2
        self.kinds.append("relu")
        return None

    def avgpool_prepare(self, m, k, stride, level):
        C, H, W, grid, dil, block = m
        self.kinds.append("pool")
        return (C, (H - k) // stride + 1, (W - k) // stride + 1, grid, dil * stride, block)

    def fc_prepare(self, m, W, level, scale, bias=None):
        F.Context._fc_weights(m, W, bias)
        self.kinds.append("fc")
        return (1, 1, W.shape[0], W.shape[0], 1, W.shape[0])

    @staticmethod
    def layer_out_map(layer):
        return layer


def test_layer_chain_shapes():
    w = lenet.weights(synth.SEED_BASE + 2)
    net = lenet.EncryptedLeNet(_ShapeCtx(), w, [2.0] * 4, lenet.levels() + 2, 2.0 ** 40)
    assert net.ctx.kinds == ["conv", "relu", "pool"] * 2 + ["fc", "relu", "fc", "relu", "fc"]
    assert net.out_level == 2
