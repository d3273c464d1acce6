"""LeNet-5 encrypted inference on the library's packed layers (the paper's
LeNet-5 of Appendix A: conv 5x5 1->6, ReLU, average pooling 2/2, conv 5x5 6->16,
ReLU, average pooling 2/2, FC 256->120, ReLU, FC 120->84, ReLU, FC 84->10).

Every layer is a C-ABI layer of the library (fheon_conv_prepare,
fheon_relu_prepare, fheon_avgpool_prepare, fheon_fc_prepare) applied with
fheon_layer_apply; this module only holds the architecture, seeded random-init
weights, the FP64 forward pass used to choose each ReLU's input bound beta
(Alg. 4 leaves beta to an analysis of the data), and the packing of inputs.

Packing: the 28x28 input in the first 784 slots, channel c of every feature
map in the block at c * 784 on the 28-wide grid; pooling leaves its outputs
at stride-aligned slots (dilation 2, then 4) instead of compacting them.
"""
import numpy as np

from . import fheon as F
from . import synth

GRID, BLOCK = 28, 784
RELU_DEGREE = 59
# (out, in, k) of the two convolutions and (out, in) of the three FC layers
CONVS = [(6, 1, 5), (16, 6, 5)]
FCS = [(120, 256), (84, 120), (10, 84)]
# levels each layer uses (a ReLU: the series' depth, + 1 for the mask when beta > 1)
DEPTH = {"conv": 1, "pool": 1, "fc": 1}


def relu_depth(beta):
    return F.cheb_depth(RELU_DEGREE) + (1 if beta > 1.0 else 0)


def levels():
    """The most levels the network uses (every ReLU with its mask)."""
    return 2 * DEPTH["conv"] + 2 * DEPTH["pool"] + 3 * DEPTH["fc"] + 4 * relu_depth(2.0)


def weights(seed):
    """Random-init FP64 weights (uniform with bound 1/sqrt(fan_in), the usual
    default initialisation of conv and linear layers)."""
    g = synth.rng(seed, 500)
    out = {}
    for i, (f, c, k) in enumerate(CONVS):
        b = 1.0 / np.sqrt(c * k * k)
        out["conv%d" % i] = (g.uniform(-b, b, (f, c, k, k)), g.uniform(-b, b, f))
    for i, (m, n) in enumerate(FCS):
        b = 1.0 / np.sqrt(n)
        out["fc%d" % i] = (g.uniform(-b, b, (m, n)), g.uniform(-b, b, m))
    return out


def _conv(X, K, b):
    C, H, W = X.shape
    F, _, k, _ = K.shape
    Ho, Wo = H - k + 1, W - k + 1
    Y = np.zeros((F, Ho, Wo))
    for x in range(k):
        for y in range(k):
            Y += np.einsum("fc,chw->fhw", K[:, :, x, y], X[:, x:x + Ho, y:y + Wo])
    return Y + b[:, None, None]


def _pool(X):
    C, H, W = X.shape
    return X.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def forward_fp64(X, w, relu=lambda v: np.maximum(v, 0.0), record=None):
    """FP64 forward pass of one 1x28x28 input; `record` collects the inputs of
    the four ReLUs."""
    def act(v):
        if record is not None:
            record.append(v)
        return relu(v)
    h = _pool(act(_conv(X, *w["conv0"])))
    h = _pool(act(_conv(h, *w["conv1"])))
    h = h.reshape(-1)
    for i in range(3):
        W, b = w["fc%d" % i]
        h = W @ h + b
        if i < 2:
            h = act(h)
    return h


def relu_bounds(inputs, w, margin=1.5):
    """beta of each ReLU: margin x the largest |input| over the calibration inputs."""
    peaks = np.zeros(4)
    for X in inputs:
        rec = []
        forward_fp64(X, w, record=rec)
        peaks = np.maximum(peaks, [np.max(np.abs(r)) for r in rec])
    return [float(max(1.0, margin * p)) for p in peaks]


def pack_input(X, nslots):
    v = np.zeros(nslots)
    v[:784] = np.asarray(X, dtype=np.float64).reshape(-1)
    return v


class EncryptedLeNet:
    """The layers of LeNet-5 prepared on a context (from level `level`)."""

    def __init__(self, ctx, w, betas, level, scale):
        self.ctx = ctx
        self.layers = []
        lv = level
        m = (1, 28, 28, GRID, 1, BLOCK)
        for i in range(2):
            K, b = w["conv%d" % i]
            conv = ctx.conv_prepare(m, K, 0, lv, scale, bias=b)
            m = ctx.layer_out_map(conv)
            lv -= DEPTH["conv"]
            relu = ctx.relu_prepare(betas[i], RELU_DEGREE, m[0] * m[5], lv)
            lv -= relu_depth(betas[i])
            pool = ctx.avgpool_prepare(m, 2, 2, lv)
            m = ctx.layer_out_map(pool)
            lv -= DEPTH["pool"]
            self.layers += [conv, relu, pool]
        for i in range(3):
            W, b = w["fc%d" % i]
            fc = ctx.fc_prepare(m, W, lv, scale, bias=b)
            m = ctx.layer_out_map(fc)
            lv -= DEPTH["fc"]
            self.layers.append(fc)
            if i < 2:
                self.layers.append(ctx.relu_prepare(betas[2 + i], RELU_DEGREE, m[2], lv))
                lv -= relu_depth(betas[2 + i])
        self.out_level = lv

    def rotation_steps(self):
        st = set()
        for layer in self.layers:
            st.update(self.ctx.layer_rotation_steps(layer))
        return sorted(st)

    def forward(self, ct):
        for layer in self.layers:
            ct = self.ctx.layer_apply(layer, ct)
        return ct

    def forward_batch(self, cts):
        """Several inputs at once: each layer applied to the whole batch in one
        call (fheon_layer_apply_batch), so the rotations of every input share
        launches; each output is the one forward() gives its input."""
        for layer in self.layers:
            cts = self.ctx.layer_apply_batch(layer, cts)
        return cts

    def forward_graph(self, ct):
        """The same layers replayed as CUDA graphs on fixed buffers: the input is
        copied into a staging ciphertext, each layer writes its own output
        buffer (the context's stream must be a created stream).  Returns a new
        ciphertext holding the output."""
        ctx = self.ctx
        if not hasattr(self, "_bufs"):
            self._bufs = [ctx.ct_create(1) for _ in range(len(self.layers) + 1)]
        ctx.drop_level(ct, ctx.ct_info(ct)[0], out=self._bufs[0])
        for i, layer in enumerate(self.layers):
            ctx.layer_apply_graph(layer, self._bufs[i], self._bufs[i + 1])
        y = self._bufs[-1]
        return ctx.drop_level(y, ctx.ct_info(y)[0])
