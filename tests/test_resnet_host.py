"""ResNet-20 host side: the package's FP64 forward pass (used to choose the
ReLU bounds) against the oracle's plain-layer network, the slot maps, and the
level plan of the encrypted network on a stand-in context that computes only
levels and maps (every layer is prepared at the level its input has) and
passes every kernel and weight matrix through the binding's own size checks."""
import numpy as np
import pytest

from oracle import fheon as OF
from paper_2510_03996_gb300 import fheon as F
from paper_2510_03996_gb300 import resnet as R
from paper_2510_03996_gb300 import synth

MINI = dict(img=8, in_ch=3, chans=(2, 4, 8), blocks=1, classes=10)


@pytest.mark.parametrize("arch", [MINI, dict(MINI, blocks=2)])
def test_fp64_forward_matches_the_oracle(arch):
    w = R.weights(0xC0, arch)
    X = synth.image(0xC1, 0, (3, arch["img"], arch["img"]), dist="normal")
    a = R.forward_fp64(X, w, arch)
    b = OF.resnet_fp64(X, w, arch["chans"], arch["blocks"])
    assert np.max(np.abs(a - b)) < 1e-10
    betas = R.relu_bounds([X], w, arch)
    assert len(betas) == R.n_relus(arch) == 1 + 6 * arch["blocks"]
    a = R.forward_fp64(X, w, arch, relu=lambda v, i: OF.relu_fp64(v, betas[i]))
    b = OF.resnet_fp64(X, w, arch["chans"], arch["blocks"], betas=betas)
    assert np.max(np.abs(a - b)) < 1e-9


def test_full_size_maps_fit_the_slots():
    n = 1 << 15
    for name, (C, H, W, grid, dil, block) in R.maps(R.FULL).items():
        assert C * block <= n, name
        assert dil * ((H - 1) * grid + (W - 1)) < block, name
    assert R.n_relus(R.FULL) == 19


class _Layer:
    def __init__(self, kind, level, out_map=None):
        self.kind, self.level, self.out_map = kind, level, out_map


class FakeCtx:
    """Levels and maps only: records every prepare call."""
    L = 32
    N = 1 << 16

    def __init__(self):
        self.calls = []

    def bootstrap_prepare(self, scale, params=None):
        return _Layer("boot", None, (params.slots, params.unmasked) if params is not None else (0, 0))

    def boot_params_default(self):
        return F.fheon_boot_params(3, 3, 512, 27, 9, 0, 0)

    def bootstrap_info(self, layer):
        return 11, 2.0 ** 40

    def conv_prepare(self, m, K, pad, level, scale, bias=None, stride=1):
        F.Context._conv_weights(m, K, bias)
        C, H, W, grid, dil, block = m
        Fo, _, k, _ = K.shape
        Ho, Wo = (H + 2 * pad - k) // stride + 1, (W + 2 * pad - k) // stride + 1
        self.calls.append(("conv", level))
        return _Layer("conv", level, (Fo, Ho, Wo, grid, dil * stride, block))

    def cheb_prepare(self, coeffs, level):
        assert level > 7
        self.calls.append(("series", level))
        return _Layer("series", level)

    def repack_prepare(self, a, b, level):
        assert a[:3] == b[:3]
        self.calls.append(("repack", level))
        return _Layer("repack", level, b)

    def global_avgpool_prepare(self, m, level):
        self.calls.append(("pool", level))
        C, H, W, grid, dil, block = m
        return _Layer("pool", level, (C, 1, 1, grid, dil * H, block))

    def fc_prepare(self, m, W, level, scale, bias=None):
        F.Context._fc_weights(m, W, bias)
        self.calls.append(("fc", level))
        return _Layer("fc", level, (1, 1, W.shape[0], W.shape[0], 1, W.shape[0]))

    @staticmethod
    def layer_out_map(layer):
        return layer.out_map


def test_level_plan_full_size():
    w = R.weights(0xC2, R.FULL)
    net = R.EncryptedResNet(FakeCtx(), w, [2.0] * R.n_relus(R.FULL), 2.0 ** 40)
    assert net.n_boot == 18 and net.in_level == 11
    assert net.out_level >= 1
    # every bootstrap input and every layer sits at a level >= 1
    levels = [c[1] for c in net.ctx.calls]
    assert min(levels) >= 2
    # stage 2's map compacted once, on the residual path and on the shortcut
    assert [c[0] for c in net.ctx.calls].count("repack") == 4
    kinds = [op[0] for op in net.plan]
    assert kinds.count("boot") == 18 and kinds.count("add") == 9


def test_bootstraps_only_where_levels_run_out():
    """With 17 levels after a bootstrap, two ReLUs and their convolutions fit
    between bootstraps: 9 instead of 18, and every layer still at level >= 2."""
    class Deep(FakeCtx):
        def bootstrap_info(self, layer):
            return 17, 2.0 ** 40
    net = R.EncryptedResNet(Deep(), R.weights(0xC3, R.FULL), [2.0] * R.n_relus(R.FULL), 2.0 ** 40)
    assert net.n_boot == 9 and net.out_level >= 1
    assert min(c[1] for c in net.ctx.calls) >= 2
    # every bootstrap input within slots [0, N/4) takes the sparse bootstrap:
    # unmasked where it is a convolution's output (zero outside its map: here
    # the second ReLU of the two blocks with a convolution on the shortcut,
    # one of them at level 1), masked otherwise (its input at level >= 2)
    kinds = [op[2].out_map for op in net.plan if op[0] == "boot"]
    assert all(k[0] == Deep.N // 4 for k in kinds)
    assert kinds.count((Deep.N // 4, 1)) == 2 and kinds.count((Deep.N // 4, 0)) == 7
    full = R.EncryptedResNet(Deep(), R.weights(0xC3, R.FULL), [2.0] * R.n_relus(R.FULL), 2.0 ** 40, sparse=False)
    assert full.n_boot == 9 and all(op[2].out_map == (0, 0) for op in full.plan if op[0] == "boot")


def test_reduced_network_plan():
    """The reduced network (one block per stage) on the test contexts' level
    11: six bootstraps, one repack pair, every layer at level >= 2."""
    net = R.EncryptedResNet(FakeCtx(), R.weights(0xC4, MINI), [2.0] * R.n_relus(MINI), 2.0 ** 40, MINI)
    assert net.n_boot == 6 and net.in_level == 11
    kinds = [op[0] for op in net.plan]
    assert kinds.count("add") == 3 and kinds.count("scale") == 1
    assert [c[0] for c in net.ctx.calls].count("repack") == 4
    assert min(c[1] for c in net.ctx.calls) >= 2 and net.out_level >= 1
