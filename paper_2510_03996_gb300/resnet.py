"""ResNet-20 encrypted inference with bootstrapping on the library's layers
(the paper's ResNet-20 of Appendix A: a 3x3 conv 3->16 and ReLU, three stages of
three residual blocks with 16, 32 and 64 channels, the first block of stages
2 and 3 with stride 2 and a 1x1 stride-2 convolution on its shortcut, global
average pooling and FC 64->10).

Every step is a C-ABI call of the library: convolutions (fheon_conv_prepare),
the ReLU's Chebyshev series (fheon_cheb_prepare with fheon_relu_coeffs),
bootstrapping (fheon_bootstrap_prepare), the one repacking of the feature map
(fheon_repack_prepare), global pooling and FC; this module holds the
architecture, seeded random-init weights, the FP64 forward pass that sets
each ReLU's input bound beta (Alg. 4 leaves beta to an analysis of the data)
and the level plan.

Placement of bootstraps: before a ReLU exactly when the levels left would
not carry its series and the layers up to the next ReLU's input with one
level to spare (the paper bootstraps before every ReLU but the first two; a
context with 16 levels of layers after a bootstrap needs one every other
ReLU).  Inputs are encrypted at the bootstrap's output level, so the first
ReLU runs without one.  The convolution in front of a ReLU carries the
ReLU's 1/beta in its weights, so its output -- the bootstrap's input -- lies
in [-1, 1]; the identity shortcut of a block is scaled by 1/beta with one
constant product on its own (shallower) path.  After a bootstrap the level
is B = L - (bootstrap depth); the ReLU series takes 6 levels
(fheon_cheb_depth(59)), a convolution one, the repacking two (in-block
compaction, then block compaction), global pooling and FC one each: the
deepest stretch between bootstraps -- series, the stage-2 stride-2
convolution, the two repacks -- needs B >= 10.

Packing: channel c of a map in the block at c * block on a grid of row
stride `grid`; stride-2 layers leave their outputs at dilated positions
(fheon_map dil 2).  Stage 2's map is compacted once, in its first block
right after the strided convolutions (on the residual path and on the
shortcut), so that every map from there on -- and stage 3's 64 channels --
fits slots [0, N/4).  A bootstrap of such a map is the sparse one (one
EvalMod instead of two); one whose input arrives at level 1 (the sparse
bootstrap's mask needs a level) is the full one.
"""
import numpy as np

from . import fheon as F
from . import synth

RELU_DEGREE = 59

FULL = dict(img=32, in_ch=3, chans=(16, 32, 64), blocks=3, classes=10)


def blocks(arch):
    """(stage, block, in_ch, out_ch, stride) of every residual block."""
    out = []
    cin = arch["chans"][0]
    for s, c in enumerate(arch["chans"]):
        for b in range(arch["blocks"]):
            stride = 2 if (s > 0 and b == 0) else 1
            out.append((s, b, cin, c, stride))
            cin = c
    return out


def weights(seed, arch=FULL):
    """Random-init FP64 weights: normal with standard deviation sqrt(2 / fan_in)
    (batch normalisation folded into them, as the paper does after training),
    small biases; the second conv of each block scaled by 1/2 so that the
    residual sums stay bounded."""
    g = synth.rng(seed, 600)
    w = {}

    def conv(name, f, c, k, gain=1.0):
        w[name] = (g.normal(0.0, gain * np.sqrt(2.0 / (c * k * k)), (f, c, k, k)), g.normal(0.0, 0.05, f))

    conv("conv0", arch["chans"][0], arch["in_ch"], 3)
    for s, b, ci, co, st in blocks(arch):
        conv("s%db%d_a" % (s, b), co, ci, 3)
        conv("s%db%d_b" % (s, b), co, co, 3, gain=0.5)
        if st == 2:
            conv("s%db%d_sc" % (s, b), co, ci, 1)
    c = arch["chans"][-1]
    w["fc"] = (g.uniform(-1.0 / np.sqrt(c), 1.0 / np.sqrt(c), (arch["classes"], c)), g.normal(0.0, 0.05, arch["classes"]))
    return w


def conv_fp64(X, K, b, stride=1, pad=1):
    C, H, W = X.shape
    Fo, _, k, _ = K.shape
    Xp = np.zeros((C, H + 2 * pad, W + 2 * pad))
    Xp[:, pad:pad + H, pad:pad + W] = X
    Ho, Wo = (H + 2 * pad - k) // stride + 1, (W + 2 * pad - k) // stride + 1
    Y = np.zeros((Fo, Ho, Wo))
    for x in range(k):
        for y in range(k):
            Y += np.einsum("fc,chw->fhw", K[:, :, x, y],
                           Xp[:, x:x + stride * (Ho - 1) + 1:stride, y:y + stride * (Wo - 1) + 1:stride])
    return Y + b[:, None, None]


def forward_fp64(X, w, arch=FULL, relu=None, record=None):
    """FP64 forward pass of one input; relu(v, i) is the i-th activation (default
    max(0, v)); `record` collects the ReLU inputs in order."""
    idx = [0]

    def act(v):
        if record is not None:
            record.append(v)
        i = idx[0]
        idx[0] += 1
        return np.maximum(v, 0.0) if relu is None else relu(v, i)

    h = act(conv_fp64(X, *w["conv0"]))
    for s, b, ci, co, st in blocks(arch):
        name = "s%db%d" % (s, b)
        t = act(conv_fp64(h, *w[name + "_a"], stride=st))
        t = conv_fp64(t, *w[name + "_b"])
        sc = conv_fp64(h, *w[name + "_sc"], stride=2, pad=0) if st == 2 else h
        h = act(t + sc)
    h = h.mean(axis=(1, 2))
    W, bias = w["fc"]
    return W @ h + bias


def relu_bounds(inputs, w, arch=FULL, margin=1.5):
    """beta of each ReLU: margin x the largest |input| over the calibration inputs."""
    peaks = None
    for X in inputs:
        rec = []
        forward_fp64(X, w, arch, record=rec)
        p = np.array([np.max(np.abs(r)) for r in rec])
        peaks = p if peaks is None else np.maximum(peaks, p)
    return [float(max(1.0, margin * p)) for p in peaks]


def n_relus(arch=FULL):
    return 1 + 2 * len(blocks(arch))


def maps(arch=FULL):
    """Slot maps (C, H, W, grid, dil, block): the input, stage 1, stage 2 as
    the stride leaves it, stage 2 compacted within its blocks, then compacted,
    stage 3 as the stride leaves it."""
    n = arch["img"]
    c1, c2, c3 = arch["chans"]
    blk = n * n
    return dict(input=(arch["in_ch"], n, n, n, 1, blk), s0=(c1, n, n, n, 1, blk),
                s1=(c2, n // 2, n // 2, n, 2, blk), s1_rows=(c2, n // 2, n // 2, n // 2, 1, blk),
                s1_packed=(c2, n // 2, n // 2, n // 2, 1, blk // 4),
                s2=(c3, n // 4, n // 4, n // 2, 2, blk // 4))


def pack_input(X, nslots, arch=FULL):
    m = maps(arch)["input"]
    C, H, W, grid, dil, block = m
    v = np.zeros(nslots)
    for c in range(C):
        for i in range(H):
            for j in range(W):
                v[c * block + dil * (i * grid + j)] = X[c, i, j]
    return v


class EncryptedResNet:
    """The layers of the network prepared on a context whose bootstrap leaves
    level B >= 10, for inputs at level B (`in_level`) at the context's scale.

    forward(ct) runs: conv0 (x 1/beta_0) -> series_0 -> per block: conv_a
    (x 1/beta) -> [bootstrap] -> series -> conv_b (x 1/beta') + shortcut
    (identity times 1/beta' by a constant product, or the 1x1 stride-2 conv
    x 1/beta') -> [bootstrap] -> series; the two repacks after stage 2; global
    pooling; FC.  The first ReLU runs without a bootstrap."""

    def __init__(self, ctx, w, betas, scale, arch=FULL, boot_params=None, sparse=True):
        self.ctx, self.w, self.betas, self.scale, self.arch = ctx, w, list(betas), float(scale), arch
        self.L = ctx.L
        self.nslots = ctx.N // 2
        self.sparse = bool(sparse)
        self._boots = {}
        # the bootstrap of feature maps within slots [0, N/4) (sparse: one
        # EvalMod), and the full one for maps beyond
        self.boot = self._boot(self.nslots // 2 if self.sparse else 0, boot_params)
        self.B = ctx.bootstrap_info(self.boot)[0]
        if self.B < 10:
            raise ValueError("the bootstrap leaves level %d; the network needs 10" % self.B)
        self._boot_params = boot_params
        self.mp = maps(arch)
        self.layers = {}
        self._series = {}
        self.plan = []  # (op, args) in order: the forward pass
        self.n_boot = 0
        self._build()

    # -- preparation -------------------------------------------------------
    def _boot(self, slots, params=None, unmasked=False):
        key = (slots, bool(unmasked))
        if key not in self._boots:
            p = None
            if slots or params is not None:
                p = params if params is not None else self.ctx.boot_params_default()
                p = type(p).from_buffer_copy(p)
                p.slots = slots
                p.unmasked = 1 if unmasked else 0
            self._boots[key] = self.ctx.bootstrap_prepare(self.scale, p)
        return self._boots[key]

    def boot_layers(self):
        """The bootstrap layers the plan uses."""
        return list(self._boots.values())

    def _series_at(self, beta, level):
        key = (beta, level)
        if key not in self._series:
            self._series[key] = self.ctx.cheb_prepare(F.relu_coeffs(beta, RELU_DEGREE), level)
        return self._series[key]

    def _conv(self, name, m, level, beta, stride=1, pad=1):
        K, b = self.w[name]
        layer = self.ctx.conv_prepare(m, K / beta, pad, level, self.scale, bias=b / beta, stride=stride)
        self.layers[name] = layer
        return layer, self.ctx.layer_out_map(layer)

    def _compact(self, reg, m, lv, tag):
        """Stage 2's strided map into its compact layout (rows and columns
        within the blocks, then the blocks: two repack layers, two levels)."""
        mp = self.mp
        rp1 = self.ctx.repack_prepare(m, mp["s1_rows"], lv)
        rp2 = self.ctx.repack_prepare(mp["s1_rows"], mp["s1_packed"], lv - 1)
        self.layers["repack1" + tag], self.layers["repack2" + tag] = rp1, rp2
        self.plan += [("layer", rp1, reg, reg), ("layer", rp2, reg, reg)]
        return lv - 2

    def _build(self):
        # registers: x = the current feature map (a block's input and output),
        # h = the residual branch, s = the shortcut
        ctx, mp, betas = self.ctx, self.mp, self.betas
        r = 0  # ReLU index
        lv = self.in_level = self.B
        m = mp["input"]
        conv, m = self._conv("conv0", m, lv, betas[r])
        self.plan.append(("layer", conv, "x", "h"))
        lv = self._relu(r, lv - 1, "h", "x", after=1, m=m, clean=True)
        r += 1
        bl = blocks(self.arch)
        for bi, (s, b, ci, co, st) in enumerate(bl):
            name = "s%db%d" % (s, b)
            # stage 2's first block compacts its strided map (both paths)
            # before its first ReLU: levels between this block's last ReLU and
            # the next ReLU's input are the next conv (and those two repacks),
            # or pooling and FC
            compact = s == 1 and b == 0
            nxt = bl[bi + 1] if bi + 1 < len(bl) else None
            after_last = 2 if nxt is None else (3 if (nxt[0] == 1 and nxt[1] == 0) else 1)
            x_level, x_map = lv, m
            conv, ma = self._conv(name + "_a", m, lv, betas[r], stride=st)
            self.plan.append(("layer", conv, "x", "h"))
            lv -= 1
            if compact:
                lv = self._compact("h", ma, lv, "")
                ma = mp["s1_packed"]
            lv = self._relu(r, lv, "h", "h", after=1, m=ma, clean=True)
            r += 1
            conv, mb = self._conv(name + "_b", ma, lv, betas[r])
            self.plan.append(("layer", conv, "h", "h"))
            lv -= 1
            if st == 2:
                sc, msc = self._conv(name + "_sc", x_map, x_level, betas[r], stride=2, pad=0)
                self.plan.append(("layer", sc, "x", "s"))
                sl = x_level - 1
                if compact:
                    sl = self._compact("s", msc, sl, "_sc")
                    msc = mp["s1_packed"]
                assert tuple(msc) == tuple(mb), (msc, mb)
            else:
                self.plan.append(("scale", 1.0 / betas[r], "x", "s"))
                sl = x_level - 1
            lv = min(lv, sl)
            self.plan.append(("add", lv, "h", "s", "h"))
            # a convolution's output is zero outside its map; an identity
            # shortcut carries the previous ReLU's values there
            lv = self._relu(r, lv, "h", "x", after=after_last, m=mb, clean=st == 2)
            r += 1
            m = mb
        # global average pooling and FC
        pool = ctx.global_avgpool_prepare(m, lv)
        self.layers["pool"] = pool
        self.plan.append(("layer", pool, "x", "x"))
        lv -= 1
        W, bias = self.w["fc"]
        fc = ctx.fc_prepare(ctx.layer_out_map(pool), W, lv, self.scale, bias=bias)
        self.layers["fc"] = fc
        self.plan.append(("layer", fc, "x", "x"))
        lv -= 1
        self.out_level = lv
        assert r == len(betas) == n_relus(self.arch)

    def _relu(self, r, lv, src, dst, after, m, clean=False):
        """The r-th ReLU of register src (at level lv, already scaled by
        1/beta_r, feature map m; `clean`: zero outside the map) into register
        dst; bootstrapped first when the levels left would not carry the
        series and the `after` levels up to the next ReLU's input with one
        level to spare.  A map within slots [0, N/4) takes the sparse
        bootstrap: unmasked when the input is clean, masked when it is at
        level 2 or more (the mask takes a level); any other the full one.
        Returns the level after it."""
        depth = F.cheb_depth(RELU_DEGREE)
        if lv - depth - after < 1:
            C, H, W, grid, dil, block = m
            fits = self.sparse and C * block <= self.nslots // 2 and (clean or lv >= 2)
            layer = self._boot(self.nslots // 2 if fits else 0, self._boot_params, unmasked=fits and clean)
            self.plan.append(("boot", src, layer))
            self.n_boot += 1
            lv = self.B
        self.plan.append(("layer", self._series_at(self.betas[r], lv), src, dst))
        return lv - depth

    def program(self):
        """The plan as model-program steps (fheon_step tuples) over registers
        x = 0, h = 1, s = 2, for fheon_model_create_program."""
        R = {"x": 0, "h": 1, "s": 2}
        F_ = F
        out = []
        for op in self.plan:
            if op[0] == "layer":
                out.append((F_.STEP_LAYER, R[op[2]], 0, R[op[3]], 0, op[1], 0.0))
            elif op[0] == "scale":
                out.append((F_.STEP_SCALE, R[op[2]], 0, R[op[3]], 0, None, op[1]))
            elif op[0] == "add":
                out.append((F_.STEP_ADD, R[op[2]], R[op[3]], R[op[4]], op[1], None, 0.0))
            elif op[0] == "boot":
                out.append((F_.STEP_LAYER, R[op[1]], 0, R[op[1]], 0, op[2], 0.0))
        return out

    def model(self):
        """The network as a native model (fheon_model_run, the server)."""
        return self.ctx.model_program(self.program(), 3, self.scale)

    def rotation_steps(self):
        st = set()
        for layer in self.layers.values():
            st.update(self.ctx.layer_rotation_steps(layer))
        return sorted(st)

    def keygen(self, sk):
        ctx = self.ctx
        ctx.relinkeygen(sk)
        for b in self.boot_layers():
            ctx.bootstrap_keygen(sk, b)
        ctx.galois_keygen(sk, sorted({ctx.galois_elt(s) for s in self.rotation_steps()}))

    # -- inference ---------------------------------------------------------
    def forward(self, ct):
        ctx = self.ctx
        reg = {"x": ct}
        for op in self.plan:
            kind = op[0]
            if kind == "layer":
                _, layer, src, dst = op
                reg[dst] = ctx.layer_apply(layer, reg[src])
            elif kind == "scale":
                _, c, src, dst = op
                reg[dst] = ctx.mul_const_rescale(reg[src], c, self.scale)
            elif kind == "add":
                _, lv, a, b, dst = op
                A, Bc = (ctx.drop_level(reg[k], lv) if ctx.ct_info(reg[k])[0] > lv else reg[k] for k in (a, b))
                reg[dst] = ctx.add(A, Bc)
            elif kind == "boot":
                reg[op[1]] = ctx.layer_apply(op[2], reg[op[1]])
        return reg["x"]

    def forward_batch(self, cts):
        """Several inputs through the same plan at once: every layer (bootstraps
        included) applied to the whole batch in one call (fheon_layer_apply_batch),
        so their rotations, products and series share launches; each output is
        the one forward() gives its input."""
        ctx = self.ctx
        reg = {"x": list(cts)}
        for op in self.plan:
            kind = op[0]
            if kind == "layer":
                _, layer, src, dst = op
                reg[dst] = ctx.layer_apply_batch(layer, reg[src])
            elif kind == "scale":
                _, c, src, dst = op
                reg[dst] = [ctx.mul_const_rescale(x, c, self.scale) for x in reg[src]]
            elif kind == "add":
                _, lv, a, b, dst = op
                out = []
                for A, Bc in zip(reg[a], reg[b]):
                    A = ctx.drop_level(A, lv) if ctx.ct_info(A)[0] > lv else A
                    Bc = ctx.drop_level(Bc, lv) if ctx.ct_info(Bc)[0] > lv else Bc
                    out.append(ctx.add(A, Bc))
                reg[dst] = out
            elif kind == "boot":
                reg[op[1]] = ctx.layer_apply_batch(op[2], reg[op[1]])
        return reg["x"]

    def forward_graph(self, ct):
        """The same plan with every layer (bootstraps included) replayed as a
        CUDA graph on fixed buffers: the input is copied into a staging
        ciphertext and every step writes its own buffer (the context's stream
        must be a created stream).  Returns a new ciphertext holding the
        output, bit for bit the one forward() gives."""
        ctx = self.ctx
        if not hasattr(self, "_bufs"):
            self._bufs = [ctx.ct_create(1) for _ in range(3 * len(self.plan) + 1)]
        bufs = self._bufs
        ctx.drop_level(ct, ctx.ct_info(ct)[0], out=bufs[-1])
        reg = {"x": bufs[-1]}
        for k, op in enumerate(self.plan):
            out = bufs[3 * k]
            kind = op[0]
            if kind == "layer":
                _, layer, src, dst = op
                reg[dst] = ctx.layer_apply_graph(layer, reg[src], out)
            elif kind == "scale":
                _, c, src, dst = op
                reg[dst] = ctx.mul_const_rescale(reg[src], c, self.scale, out=out)
            elif kind == "add":
                _, lv, a, b, dst = op
                A = ctx.drop_level(reg[a], lv, out=bufs[3 * k + 1])
                Bc = ctx.drop_level(reg[b], lv, out=bufs[3 * k + 2])
                reg[dst] = ctx.add(A, Bc, out=out)
            elif kind == "boot":
                reg[op[1]] = ctx.layer_apply_graph(op[2], reg[op[1]], out)
        y = reg["x"]
        return ctx.drop_level(y, ctx.ct_info(y)[0])
