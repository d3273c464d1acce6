"""FHEON's packed layers, restated for the oracle, plus the FP64 plaintext CNN.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

Slot conventions (paper Sec. 4.1, input flattening): a (C, H, W) tensor sits
at slot c*H*W + h*W + w.  Rot_r moves slot i+r to slot i (r > 0 rotates left),
which is the reading under which the nine masks of Algorithm 3 match the
rotations of Algorithm 1.
"""
import numpy as np

from . import ckks


# ------------------------------------------------------------- FP64 CNN
def conv2d_fp64(X, K, b=None, stride=1, pad=0):
    """Convolution as the paper's Sec. 4.1 equation states it (cross-correlation:
    Y[f,h,w] = sum_c sum_i sum_j X[c, h*s+i, w*s+j] K[f,c,i,j] + b_f) on the
    zero-padded input; output size (H + 2p - k)/s + 1 per side."""
    X = np.asarray(X, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    C, H, W = X.shape
    F, C2, kh, kw = K.shape
    assert C == C2
    Xp = np.zeros((C, H + 2 * pad, W + 2 * pad))
    Xp[:, pad:pad + H, pad:pad + W] = X
    Ho = (H + 2 * pad - kh) // stride + 1
    Wo = (W + 2 * pad - kw) // stride + 1
    Y = np.zeros((F, Ho, Wo))
    for f in range(F):
        for h in range(Ho):
            for w in range(Wo):
                Y[f, h, w] = np.sum(Xp[:, h * stride:h * stride + kh, w * stride:w * stride + kw] * K[f])
        if b is not None:
            Y[f] += b[f]
    return Y


def avgpool_fp64(X, k, stride):
    """Average pooling, paper Sec. 4.4 equation: mean over each k x k window."""
    C, H, W = X.shape
    Ho, Wo = (H - k) // stride + 1, (W - k) // stride + 1
    Y = np.zeros((C, Ho, Wo))
    for c in range(C):
        for i in range(Ho):
            for j in range(Wo):
                Y[c, i, j] = X[c, i * stride:i * stride + k, j * stride:j * stride + k].mean()
    return Y


# ------------------------------------------------------------- masks
def build_mask(sp, ep, w, m, C):
    """Algorithm 2 (build_mask) as written; its undefined loop bound t is read as C."""
    mask = [0.0] * sp
    while len(mask) < m - ep:
        mask.extend([1.0] * w)
        mask.append(0.0)
    while len(mask) > m:
        mask.pop()
    while len(mask) < m:
        mask.append(0.0)
    for i in range(ep):
        mask[m - i - 1] = 0.0
    tmask = []
    for _ in range(C):
        tmask.extend(mask)
    return np.array(tmask)


def algorithm3_masks(W, C):
    """The nine masks of Algorithm 3 for a W x W input with C channels (m = W^2)."""
    m = W * W
    args = [(W + 1, 0, W - 1), (W, 0, m), (W, 0, W - 1),
            (1, 0, W - 1), (0, 0, m), (0, 1, W - 1),
            (1, W - 1, W - 1), (0, W, m), (0, W + 1, W - 1)]
    return [build_mask(sp, ep, w, m, C) for sp, ep, w in args]


def taps(k):
    """Tap offsets (di, dj) of a k x k 'same' kernel, row-major: the order r_0..r_{k^2-1}
    of Algorithm 1 generalised from 3 x 3."""
    p = (k - 1) // 2
    return [(di, dj) for di in range(-p, p + 1) for dj in range(-p, p + 1)]


def tap_mask(H, W, C, di, dj):
    """Validity of tap (di, dj) at every output position, repeated for C channels:
    1 where (h+di, w+dj) lies inside the H x W input.  For k = 3 this equals the
    Algorithm 3 masks (checked by the tests)."""
    h = np.arange(H)[:, None]
    w = np.arange(W)[None, :]
    v = ((h + di >= 0) & (h + di < H) & (w + dj >= 0) & (w + dj < W)).astype(np.float64)
    return np.tile(v.reshape(-1), C)


def rot_slots(x, r):
    """Rot_r on a slot vector: slot i <- slot (i + r) mod n."""
    return np.roll(x, -r)


def special_conv_slots(x, H, W, C, K, k):
    """Slot-level special convolution ('same', stride 1, pad (k-1)/2), one output
    channel: sum over taps of mask_t * kernel value * Rot_{di*W+dj}(x), then the
    channel sum by Rot_{H*W} repeated C-1 times (Sec. 4.3), channel block 0 kept."""
    n = len(x)
    acc = np.zeros(n)
    for (di, dj) in taps(k):
        p = (k - 1) // 2
        vec = np.zeros(n)
        for c in range(C):
            vec[c * H * W:(c + 1) * H * W] = K[c, di + p, dj + p] * tap_mask(H, W, 1, di, dj)
        acc += vec * rot_slots(x, di * W + dj)
    tot = acc.copy()
    cur = acc
    for _ in range(C - 1):
        cur = rot_slots(cur, H * W)
        tot = tot + cur
    out = np.zeros(n)
    out[:H * W] = tot[:H * W]
    return out


# ------------------------------------------------------------- encrypted
def tap_vectors(n, H, W, C, K, k):
    """Per-tap weight vectors (kernel value x tap mask per channel block)."""
    p = (k - 1) // 2
    vecs = []
    for (di, dj) in taps(k):
        vec = np.zeros(n)
        for c in range(C):
            vec[c * H * W:(c + 1) * H * W] = K[c, di + p, dj + p] * tap_mask(H, W, 1, di, dj)
        vecs.append(vec)
    return vecs


def conv_rotation_steps(W, k):
    """Rotation amounts the special conv needs (one direct key per non-zero tap)."""
    return [di * W + dj for (di, dj) in taps(k) if (di, dj) != (0, 0)]


def special_conv_encrypted(ctx, ct, rotkeys, H, W, k, tap_plains, bias_plain=None, hoisted=False):
    """Encrypted special conv of one channel (C = 1), FHEON Sec. 4.3 generalised to
    k x k: r_t = Rot_{di*W+dj}(ct) with a direct key per tap, products with the
    tap plaintexts (encoded at scale q_{level-1}), summed, one rescale, bias added.
    hoisted: the tap rotations share one raising of c1 (the fast rotations of
    Sec. 2.2), as ctx.rotate_hoisted computes them.

    rotkeys: dict step -> key-switching key; tap_plains: list of evaluation-form
    plaintexts over Q_level in taps(k) order."""
    N = ctx.N
    acc = None
    steps = [di * W + dj for di, dj in taps(k) if di * W + dj != 0]
    if hoisted:
        hs = ctx.rotate_hoisted(ct, [ckks.galois_elt(r, N) for r in steps], [rotkeys[r] for r in steps])
        rots = dict(zip(steps, hs))
    for t, (di, dj) in enumerate(taps(k)):
        r = di * W + dj
        if r == 0:
            rt = ct
        elif hoisted:
            rt = rots[r]
        else:
            rt = ctx.rotate(ct, ckks.galois_elt(r, N), rotkeys[r])
        prod = ctx.mul_plain(rt, tap_plains[t])
        acc = prod if acc is None else ctx.add(acc, prod)
    out = ctx.rescale(acc)
    if bias_plain is not None:
        out = ctx.add_plain(out, bias_plain)
    return out


def encode_tap_plains(ctx, H, W, K, k, level):
    """Oracle encoding of the tap weight vectors at scale q_{level-1}."""
    n = ctx.N // 2
    C = K.shape[0]
    scale = float(ctx.q[level - 1])
    return [ctx.plain_from_coeffs(ckks.encode(v, ctx.N, scale), level)
            for v in tap_vectors(n, H, W, C, K, k)]


# ------------------------------------------------------------------ ReLU (Sec. 4.6, Alg. 4)
RELU_DEGREE = 59  # the paper's default D


def relu_cheb_coeffs(beta, D=RELU_DEGREE):
    """Chebyshev coefficients c_0..c_D of f(z) = beta * max(0, z) on [-1, 1],
    interpolated at the D+1 Chebyshev nodes (computed by the C oracle)."""
    import ctypes

    from . import _lib
    out = (ctypes.c_double * (D + 1))()
    _lib.lib().oracle_cheb_coeffs(float(beta), D, out)
    return np.array(out[:], dtype=np.float64)


def cheb_eval_fp64(c, z):
    """sum_d c_d T_d(z) in FP64 (T by its three-term recurrence)."""
    z = np.asarray(z, dtype=np.float64)
    t0, t1 = np.ones_like(z), z
    y = c[0] * t0 + (c[1] * t1 if len(c) > 1 else 0.0)
    for d in range(2, len(c)):
        t0, t1 = t1, 2.0 * z * t1 - t0
        y = y + c[d] * t1
    return y


def relu_fp64(x, beta, D=RELU_DEGREE):
    """The plaintext value of the approximate ReLU: the Chebyshev series of
    beta * max(0, z) at z = x / beta."""
    return cheb_eval_fp64(relu_cheb_coeffs(beta, D), np.asarray(x, dtype=np.float64) / beta)


def relu_mask_values(nslots, beta, n):
    """Alg. 4's scale mask: 1/beta in the first n slots, 0 elsewhere."""
    v = np.zeros(nslots)
    v[:n] = 1.0 / beta
    return v


def relu_encrypted(ctx, ct, scale, beta, D, mask_plain, rlk):
    """Alg. 4 on a ciphertext of scale `scale` (returns (ct, scale)):
    v = x * mask (rescaled; only when beta > 1), then the Chebyshev series of f
    at v.  T_1 = v; T_2h = 2 T_h^2 - 1; T_2h+1 = 2 T_h+1 T_h - T_1 (products at
    the lower operand level, rescaled; T_1 brought to the product's level and
    scale by a rescaled constant product).  Every c_d T_d (d >= 1) is rescaled
    onto `scale` at one common level and summed in order of d; c_0 is added
    last.  The output has the input's scale, at depth ceil(log2 D) + 1 (+1
    with the mask) below the input."""
    q = ctx.q
    c = relu_cheb_coeffs(beta, D)
    lev = lambda a: a.shape[1]  # noqa: E731
    v = ctx.rescale(ctx.mul_plain(ct, mask_plain)) if beta > 1 else ct
    T = {1: (v, scale)}
    for d in range(2, D + 1):
        if d % 2 == 0:
            A, sa = T[d // 2]
            prod = ctx.rescale(ctx.mul_relin(ctx.mul_int(A, 2), A, rlk))
            sc = sa * sa / float(q[lev(A) - 1])
            T[d] = (ctx.add_const(prod, -1.0, sc), sc)
        else:
            (A, sa), (B, sb) = T[(d + 1) // 2], T[(d - 1) // 2]
            lv = min(lev(A), lev(B))
            A, B = ctx.drop_level(A, lv), ctx.drop_level(B, lv)
            prod = ctx.rescale(ctx.mul_relin(ctx.mul_int(A, 2), B, rlk))
            sc = sa * sb / float(q[lv - 1])
            t1, s1 = T[1]
            neg = ctx.mul_const_rescale(ctx.drop_level(t1, lv), -1.0, sc, s1)
            T[d] = (ctx.add(prod, neg), sc)
    lstar = min(lev(T[d][0]) for d in T) - 1
    y = None
    for d in range(1, D + 1):
        A, sa = T[d]
        term = ctx.mul_const_rescale(ctx.drop_level(A, lstar + 1), c[d], scale, sa)
        y = term if y is None else ctx.add(y, term)
    return ctx.add_const(y, c[0], scale), scale
