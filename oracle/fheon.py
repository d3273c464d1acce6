"""FHEON's packed layers, restated for the oracle, plus the FP64 plaintext CNN.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

Slot conventions (paper Sec. 5.1, input flattening): a (C, H, W) tensor sits
at slot c*H*W + h*W + w.  Rot_r moves slot i+r to slot i (r > 0 rotates left),
which is the reading under which the nine masks of Algorithm 3 match the
rotations of Algorithm 1.
"""
import math

import numpy as np

from . import ckks


# ------------------------------------------------------------- FP64 CNN
def conv2d_fp64(X, K, b=None, stride=1, pad=0):
    """Convolution as the paper's Sec. 5.1 equation states it (cross-correlation:
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
    """Average pooling, paper Sec. 5.4 equation: mean over each k x k window."""
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
    channel sum by Rot_{H*W} repeated C-1 times (Sec. 5.3), channel block 0 kept."""
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
    """Encrypted special conv of one channel (C = 1), FHEON Sec. 5.3 generalised to
    k x k: r_t = Rot_{di*W+dj}(ct) with a direct key per tap, products with the
    tap plaintexts (encoded at scale q_{level-1}), summed, one rescale, bias added.
    hoisted: the tap rotations share one raising of c1 (the fast rotations of
    Sec. 3.2), as ctx.rotate_hoisted computes them.

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


# ------------------------------------------------------------------ ReLU (Sec. 5.6, Alg. 4)
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


def ps_params(D):
    """Baby-step count k = 2^ceil(log2(D+1)/2) and giant count m, the least with
    D < k 2^m, of the baby-step/giant-step (Paterson-Stockmeyer) evaluation
    of a degree-D Chebyshev series."""
    k = 1 << math.ceil(math.log2(D + 1) / 2)
    m = 0
    while k * (1 << m) <= D:
        m += 1
    return k, m


def cheb_depth(D):
    """Levels cheb_encrypted consumes for degree D: a product lands one level
    below the lower of its operands, a leaf one below the lowest baby it
    reads."""
    k, m = ps_params(D)
    dep = {1: 0}
    for d in range(2, min(k, D) + 1):
        dep[d] = max(dep[d - d // 2], dep[d // 2]) + 1
    gd = [dep[k]] if m else []
    for _ in range(1, m):
        gd.append(gd[-1] + 1)

    def leaf(deg):
        return max(dep[i] for i in range(1, max(deg, 1) + 1)) + 1

    def depth_of(deg, j):
        if j == 0:
            return leaf(deg)
        g = k << (j - 1)
        if deg < g:
            return depth_of(deg, j - 1)
        return max(max(depth_of(deg - g, j - 1), gd[j - 1]) + 1, depth_of(g - 1, j - 1))
    return depth_of(D, m)


def cheb_split(c, g):
    """p = r + q T_g for a series c of degree < 2g (from 2 T_g T_j = T_{g+j} +
    T_{g-j}): q_0 = c_g, q_j = 2 c_{g+j}; r_i = c_i (i < g) less c_{g+j} at
    i = g - j."""
    deg = len(c) - 1
    q = [c[g]] + [2.0 * c[g + j] for j in range(1, deg - g + 1)]
    r = list(c[:g])
    for j in range(1, deg - g + 1):
        r[g - j] = r[g - j] - c[g + j]
    return q, r


def ps_eval_fp64(c, z):
    """The series c at z in FP64 along the same tree as cheb_encrypted."""
    D = len(c) - 1
    k, m = ps_params(D)
    z = np.asarray(z, dtype=np.float64)
    T = {0: np.ones_like(z), 1: z}
    for d in range(2, min(k, D) + 1):
        h = d // 2
        T[d] = 2.0 * T[d - h] * T[h] - (T[1] if d % 2 else 1.0)
    G = [T[k]] if m else []
    for _ in range(1, m):
        G.append(2.0 * G[-1] * G[-1] - 1.0)

    def ev(c, j):
        deg = len(c) - 1
        if j == 0:
            return sum(c[i] * T[i] for i in range(deg + 1))
        g = k << (j - 1)
        if deg < g:
            return ev(c, j - 1)
        cq, cr = cheb_split(c, g)
        return ev(cr, j - 1) + ev(cq, j - 1) * G[j - 1]
    return ev(list(c), m)


def cheb_encrypted(ctx, v, scale, c, rlk):
    """sum_d c_d T_d(v) for a ciphertext v of scale `scale` (returns the
    ciphertext, of scale `scale`), by baby steps and giant steps:
      babies T_1..T_k (k = ps_params): T_2h = 2 T_h^2 - 1 (product at T_h's
        level, rescaled, then -1 added); T_2h+1 = 2 T_h+1 T_h - T_1 (the
        product, scale S = s_h+1 s_h at the lower operand level, plus T_1 times
        K = llround((-1 * S) / s_1), rescaled once);
      giants G_0 = T_k, G_j = 2 G_j-1^2 - 1 = T_{k 2^j};
      ev(c, j) for degree < k 2^j: a leaf (j = 0) is sum_i K_i T_i over
        T_1..T_deg at the lowest of their levels, K_i = llround(((c_i * S_t)
        * q) / s_i) for the prime q it is rescaled by, plus c_0: it lands on
        the target scale S_t.  Otherwise, with g = k 2^(j-1) and p = r + q
        T_g (cheb_split): ev(q) aimed at S_t q_p / s_G (q_p the prime of the
        product's rescale at level l_p = min(level of ev(q), level of G)),
        times G_j-1 at l_p, rescaled; plus ev(r) aimed at S_t; the two at
        the lower of their levels.
    Depth cheb_depth(D) (6 for degree 59, at most ceil(log2 D) + 1), with
    about 2 sqrt(D) + log2 D products instead of D - 1."""
    q = ctx.q
    D = len(c) - 1
    k, m = ps_params(D)
    lev = lambda a: a.shape[1]  # noqa: E731
    T = {1: (v, scale)}
    for d in range(2, min(k, D) + 1):
        (A, sa), (B, sb) = T[d - d // 2], T[d // 2]
        lv = min(lev(A), lev(B))
        A, B = ctx.drop_level(A, lv), ctx.drop_level(B, lv)
        prod = ctx.mul_relin(ctx.mul_int(A, 2), B, rlk)
        S = sa * sb
        sc = S / float(q[lv - 1])
        if d % 2 == 0:
            T[d] = (ctx.add_const(ctx.rescale(prod), -1.0, sc), sc)
        else:
            t1, s1 = T[1]
            K = ckks.llround((-1.0 * S) / s1)
            T[d] = (ctx.rescale(ctx.add(prod, ctx.mul_int(ctx.drop_level(t1, lv), K))), sc)
    G = [T[k]] if m else []
    for _ in range(1, m):
        A, sa = G[-1]
        prod = ctx.mul_relin(ctx.mul_int(A, 2), A, rlk)
        sc = (sa * sa) / float(q[lev(A) - 1])
        G.append((ctx.add_const(ctx.rescale(prod), -1.0, sc), sc))

    def leaf_level(deg):
        return min(lev(T[i][0]) for i in range(1, max(deg, 1) + 1)) - 1

    def out_level(deg, j):
        if j == 0:
            return leaf_level(deg)
        g = k << (j - 1)
        if deg < g:
            return out_level(deg, j - 1)
        return min(min(out_level(deg - g, j - 1), lev(G[j - 1][0])) - 1, out_level(g - 1, j - 1))

    def ev(c, j, St):
        deg = len(c) - 1
        if j == 0:
            lv = leaf_level(deg) + 1
            y = None
            for i in range(1, max(deg, 1) + 1):
                A, sa = T[i]
                term = ctx.mul_int(ctx.drop_level(A, lv), ctx.const_factor(lv, c[i] if i <= deg else 0.0, St, sa))
                y = term if y is None else ctx.add(y, term)
            return ctx.add_const(ctx.rescale(y), c[0], St)
        g = k << (j - 1)
        if deg < g:
            return ev(c, j - 1, St)
        cq, cr = cheb_split(c, g)
        Gc, sg = G[j - 1]
        lp = min(out_level(len(cq) - 1, j - 1), lev(Gc))
        qct = ev(cq, j - 1, (St * float(q[lp - 1])) / sg)
        prod = ctx.rescale(ctx.mul_relin(ctx.drop_level(qct, lp), ctx.drop_level(Gc, lp), rlk))
        rct = ev(cr, j - 1, St)
        lo = min(lev(prod), lev(rct))
        return ctx.add(ctx.drop_level(rct, lo), ctx.drop_level(prod, lo))

    return ev(list(c), m, scale)


def relu_encrypted(ctx, ct, scale, beta, D, mask_plain, rlk):
    """Alg. 4 on a ciphertext of scale `scale` (returns (ct, scale)):
    v = x * mask (rescaled; only when beta > 1), then the Chebyshev series of f
    at v (cheb_encrypted).  The output has the input's scale, at depth
    cheb_depth(D) (+1 with the mask) below the input."""
    c = relu_cheb_coeffs(beta, D)
    v = ctx.rescale(ctx.mul_plain(ct, mask_plain)) if beta > 1 else ct
    return cheb_encrypted(ctx, v, scale, c, rlk), scale


# ------------------------------------------------------------------ packed network layers
# Layout of a feature map (C, H, W) in the slots: channel c in the block at
# offset c * block; position (i, j) at c * block + dil * (i * grid + j), where
# `grid` is the row stride of the block's grid and `dil` the spacing of the
# valid positions (a stride-s layer multiplies it by s instead of compacting).

def map_slots(C, H, W, grid, dil, block):
    """Slot of every (c, i, j) of a (C, H, W) map, in flatten order."""
    return np.array([c * block + dil * (i * grid + j) for c in range(C) for i in range(H) for j in range(W)],
                    dtype=np.int64)


def pack_map(X, nslots, grid, dil, block):
    v = np.zeros(nslots)
    v[map_slots(*X.shape, grid, dil, block)] = np.asarray(X, dtype=np.float64).reshape(-1)
    return v


def unpack_map(v, shape, grid, dil, block):
    return np.asarray(v)[map_slots(*shape, grid, dil, block)].reshape(shape)


def conv_baby(k, C, F):
    """Baby steps B of the block shifts: the B minimising B k^2 - 1 + 2 ceil(G/B),
    G = C + F - 1 (the hoisted tap rotations, plus the giant steps counted at
    twice a hoisted rotation), the smaller on ties."""
    G = C + F - 1
    best, cost = 1, None
    for B in range(1, G + 1):
        c = k * k * B - 1 + 2 * (-(-G // B))
        if cost is None or c < cost:
            best, cost = B, c
    return best


def conv_plan(C, F, k, pad, H, W, grid, dil, block, nslots, K, stride=1, baby=None):
    """Rotation-sum plan of a convolution (Sec. 5.1 equation, zero padding
    `pad`, stride `stride`) from C to F channels.  Tap (x, y) reads the input
    at offset (x - pad, y - pad), i.e. Rot_r with r = dil*((x-pad)*grid +
    (y-pad)).  Block shift delta = f - c collects, in the block of input
    channel c, the weights K[f, c, x, y] at every output position --
    input-grid position (stride*i, stride*j), so the output dilation is
    dil*stride -- whose tap source lies inside the input; it moves to block f
    by Rot_{-delta*block}.  The shifts go by baby steps and giant steps:
    delta = a + B b (0 <= a < B = conv_baby unless `baby` is given) and
      Rot_{-delta block}(P * Rot_r(x)) = Rot_{-B b block}(Rot_{-a block}(P) * Rot_{r - a block}(x)),
    so the taps are r - a*block (a-major, then (x, y); a step shared by two
    pairs appears once, with their vectors summed) and group b shifts by
    -B*b*block with the vectors moved by a*block.  Returns (r, [(s_g, [values_t
    or None])]); all-zero plaintexts are None, groups without any are left out."""
    Ho, Wo = (H + 2 * pad - k) // stride + 1, (W + 2 * pad - k) // stride + 1
    B = conv_baby(k, C, F) if baby is None else baby
    taps = [(x, y) for x in range(k) for y in range(k)]
    # each step once: where the taps span more than a block, pairs (a, tap)
    # can share a step, and their vectors are summed (in (a, tap) order)
    r, index = [], []
    for a in range(B):
        for x, y in taps:
            st = dil * ((x - pad) * grid + (y - pad)) - a * block
            if st not in r:
                r.append(st)
            index.append(r.index(st))

    def add_vec(acc, delta, x, y, a):
        any_ = False
        for c in range(C):
            f = c + delta
            if not 0 <= f < F or K[f][c][x][y] == 0.0:
                continue
            for i in range(Ho):
                for j in range(Wo):
                    si, sj = stride * i + x - pad, stride * j + y - pad
                    if 0 <= si < H and 0 <= sj < W:
                        s_ = (c * block + dil * stride * (i * grid + j) + a * block) % nslots
                        acc[s_] = acc[s_] + K[f][c][x][y]
                        any_ = True
        return any_

    groups = []
    for b in range((-(C - 1)) // B, (F - 1) // B + 1):
        acc = [np.zeros(nslots) for _ in r]
        used = [False] * len(r)
        for a in range(B):
            delta = a + B * b
            if not -(C - 1) <= delta <= F - 1:
                continue
            for ti, (x, y) in enumerate(taps):
                t = index[a * len(taps) + ti]
                if add_vec(acc[t], delta, x, y, a):
                    used[t] = True
        vals = [v if u and np.any(v != 0.0) else None for v, u in zip(acc, used)]
        if any(v is not None for v in vals):
            groups.append((-B * b * block, vals))
    return r, groups


def avgpool_plan(C, k, stride, H, W, grid, dil, block, nslots):
    """Average pooling (Sec. 5.4): the window sum by the rotations
    r_t = dil*(x*grid + y), x, y < k, times one mask holding 1/k^2 at the
    stride-aligned outputs (the striding is the mask: the outputs stay in
    place, at spacing dil*stride).  Returns (r, [(0, [mask] * k^2)])."""
    Ho, Wo = (H - k) // stride + 1, (W - k) // stride + 1
    m = np.zeros(nslots)
    for c in range(C):
        for i in range(Ho):
            for j in range(Wo):
                m[c * block + dil * stride * (i * grid + j)] = 1.0 / (k * k)
    r = [dil * (x * grid + y) for x in range(k) for y in range(k)]
    return r, [(0, [m] * len(r))]


def fc_plan(Wmat, in_slots, nslots):
    """Fully connected layer (Sec. 5.5 equation): neuron k's weight vector at
    the input's slots (product, then the sum of all slots), and the one-hot
    vector that places the sum in slot k.  Returns ([W_k], [E_k])."""
    Wmat = np.asarray(Wmat, dtype=np.float64)
    m, n = Wmat.shape
    ws, es = [], []
    for k in range(m):
        w = np.zeros(nslots)
        w[np.asarray(in_slots)] = Wmat[k]
        e = np.zeros(nslots)
        e[k] = 1.0
        ws.append(w)
        es.append(e)
    return ws, es


def slot_sum_steps(nslots):
    """Rotate-and-add steps that leave the sum of all slots in every slot."""
    return [1 << t for t in range(int(np.log2(nslots)))]


def linear_slots(v, r, groups):
    """FP64 slot model of a rotation-sum plan (Rot_r(v) = v shifted left by r)."""
    out = np.zeros_like(v)
    for s, vals in groups:
        z = np.zeros_like(v)
        for rt, p in zip(r, vals):
            if p is not None:
                z += np.roll(v, -rt) * p
        out += np.roll(z, -s)
    return out


def fc_slots(v, ws, es):
    out = np.zeros_like(v)
    for w, e in zip(ws, es):
        out += np.sum(v * w) * e
    return out


def linear_steps(r, groups):
    """Rotation steps (keys) a rotation-sum plan uses."""
    return sorted({x for x in r if x != 0} | {s for s, _ in groups if s != 0})


def linear_encrypted(ctx, ct, r, groups, pts, keys):
    """A rotation-sum plan on a ciphertext: the tap rotations hoisted from the
    input, each group's products summed and rescaled once, moved by its own
    (plain) rotation, the groups summed in order.  pts[g][t]: plaintext or
    None (as in `groups`); keys: step -> key-switching key."""
    N = ctx.N
    steps = [x for x in r if x != 0]
    hs = ctx.rotate_hoisted(ct, [ckks.galois_elt(x, N) for x in steps], [keys[x] for x in steps])
    rot = dict(zip(steps, hs))
    rot[0] = ct
    y = None
    for (s, _), gp in zip(groups, pts):
        acc = None
        for rt, p in zip(r, gp):
            if p is not None:
                prod = ctx.mul_plain(rot[rt], p)
                acc = prod if acc is None else ctx.add(acc, prod)
        acc = ctx.rescale(acc)
        if s != 0:
            acc = ctx.rotate(acc, ckks.galois_elt(s, N), keys[s])
        y = acc if y is None else ctx.add(y, acc)
    return y


def fc_encrypted(ctx, ct, wpts, epts, keys):
    """FC plan on a ciphertext: t_k = rescale(ct * W_k); every t_k through the
    rotate-and-add slot sum; out = rescale(sum_k t_k * E_k)."""
    N = ctx.N
    ts = [ctx.rescale(ctx.mul_plain(ct, w)) for w in wpts]
    for st in slot_sum_steps(N // 2):
        g = ckks.galois_elt(st, N)
        ts = [ctx.add(t, ctx.rotate(t, g, keys[st])) for t in ts]
    y = None
    for t, e in zip(ts, epts):
        prod = ctx.mul_plain(t, e)
        y = prod if y is None else ctx.add(y, prod)
    return ctx.rescale(y)


def lenet_fp64(X, w, betas=None, D=RELU_DEGREE):
    """LeNet-5 (paper's Appendix A architecture) in FP64 from the plain layers; with
    `betas`, each ReLU is the Chebyshev series of Alg. 4 with that bound."""
    def act(v, i):
        return np.maximum(v, 0.0) if betas is None else relu_fp64(v, betas[i], D)
    h = avgpool_fp64(act(conv2d_fp64(X, w["conv0"][0], b=w["conv0"][1]), 0), 2, 2)
    h = avgpool_fp64(act(conv2d_fp64(h, w["conv1"][0], b=w["conv1"][1]), 1), 2, 2)
    h = h.reshape(-1)
    for i in range(3):
        W, b = w["fc%d" % i]
        h = W @ h + b
        if i < 2:
            h = act(h, 2 + i)
    return h


def fold_offsets(C, H, W, grid, dil, block):
    """Where the fold puts channel c inside block 0: at row offset c // dil and
    column offset c % dil of the dilation grid, so the channels interleave.
    Only when every channel fits (C <= dil^2, dil*W <= grid) and the folded
    region stays inside the block; else None (no fold).  Rot_{f_c} also moves
    every other channel c' to block c' - c, which the layer never reads."""
    if dil < 2 or C > dil * dil or dil * W > grid:
        return None
    off = [(c % dil) + grid * (c // dil) for c in range(C)]
    if max(off) + dil * ((H - 1) * grid + (W - 1)) >= block:
        return None
    return off


def fc_diag_plan(Wmat, C, H, W, grid, dil, block, nslots):
    """Fully connected layer (Sec. 5.5 equation) in diagonal form.
    Fold (when fold_offsets allows it): x' = sum_c Rot_{f_c}(x),
    f_c = c*block - off_c, brings channel c's values (zero elsewhere) to
    off_c + dil*(i*grid + j) in block 0.  Then y[k] = sum_d diag_d[k] x'[k + d] with
    diag_d[k] = W[k, t] where input t sits at slot k + d; baby-step giant-step:
    d = e_g + a (a < b, e_g = d_min + g*b), so y = sum_g Rot_{e_g}( sum_a
    Rot_{-e_g}(diag_d) * Rot_a(x') ).  Returns (fold shifts, r, groups) with the
    rotation-sum conventions of `conv_plan`."""
    Wmat = np.asarray(Wmat, dtype=np.float64)
    m, n_in = Wmat.shape
    assert n_in == C * H * W
    off = fold_offsets(C, H, W, grid, dil, block)
    fold = [c * block - off[c] for c in range(C)] if off else []
    off = off or [c * block for c in range(C)]
    slots = [off[c] + dil * (i * grid + j) for c in range(C) for i in range(H) for j in range(W)]
    assert len(set(slots)) == len(slots)
    dmin = min(slots) - (m - 1)
    dmax = max(slots)
    span = dmax - dmin + 1
    b = int(np.ceil(np.sqrt(span)))
    ng = (span + b - 1) // b
    r = list(range(b))
    groups = []
    for g in range(ng):
        e = dmin + g * b
        vals = []
        for a in range(b):
            d = e + a
            diag = np.zeros(nslots)
            for t, st in enumerate(slots):
                k = st - d
                if 0 <= k < m:
                    diag[k] = Wmat[k, t]
            vals.append(np.roll(diag, e) if np.any(diag != 0.0) else None)
        if any(v is not None for v in vals):
            groups.append((e, vals))
    return fold, r, groups


def fold_slots(v, fold):
    if not fold:
        return v
    return sum(np.roll(v, -f) for f in fold)


def fold_encrypted(ctx, ct, fold, keys):
    """x' = sum_c Rot_{f_c}(ct), the rotations hoisted from ct, summed in order."""
    if not fold:
        return ct
    N = ctx.N
    steps = [f for f in fold if f != 0]
    hs = dict(zip(steps, ctx.rotate_hoisted(ct, [ckks.galois_elt(f, N) for f in steps], [keys[f] for f in steps])))
    y = None
    for f in fold:
        t = ct if f == 0 else hs[f]
        y = t if y is None else ctx.add(y, t)
    return y


# ------------------------------------------------------------------ BSGS rotation sums and repacking
def bsgs_plan(diags, n, stride, baby=0):
    """Baby-step/giant-step form of sum_o d_o Rot_o: every offset is k*stride
    (k centred in (-M/2, M/2], M = n/stride), split as k = c*bs + t with
    0 <= t < bs; then
      out = sum_c Rot_{G_c}( sum_t Rot_{-G_c}(d_k) * Rot_{t stride}(in) ),  G_c = c bs stride.
    Returns (taps r, groups [(G_c, [vector or None per tap])]) in the
    rotation-sum form of the linear layers.  bs = `baby`, else the power of
    two with the fewest rotations (ties: the larger bs)."""
    M = n // stride
    ks = {}
    for o, d in diags.items():
        assert o % stride == 0
        k = o // stride
        if k > M // 2:
            k -= M
        if np.any(d != 0):
            ks[k] = d
    def cost(bs):
        ts = {k - (k // bs) * bs for k in ks}
        cs = {k // bs for k in ks}
        return len(ts - {0}) + len(cs - {0})
    if baby:
        bs = baby
    else:
        bs, best = 1, None
        b = 1
        while b <= M:
            c = cost(b)
            if best is None or c <= best:
                bs, best = b, c
            b *= 2
    ts = sorted({k - (k // bs) * bs for k in ks})
    r = [t * stride for t in ts]
    groups = []
    for c in sorted({k // bs for k in ks}):
        G = c * bs * stride
        vals = []
        for t in ts:
            k = c * bs + t
            vals.append(np.roll(ks[k], G) if k in ks else None)
        groups.append((G, vals))
    return r, groups


def plan_slots(v, r, groups):
    """FP64 model of a rotation-sum plan on complex slots."""
    out = np.zeros(len(v), dtype=np.complex128)
    for G, vals in groups:
        z = np.zeros(len(v), dtype=np.complex128)
        for rt, p in zip(r, vals):
            if p is not None:
                z += np.roll(v, -rt) * p
        out += np.roll(z, -G)
    return out


def repack_plan(C, H, W, src, dst, nslots):
    """A (C, H, W) map moved from layout src = (grid, dil, block) to layout
    dst in one level (striding by extraction, Sec. 5.2): out = sum_o m_o
    Rot_o(in), m_o one at every destination slot whose source is o slots
    further on; in BSGS form over the largest power-of-two stride dividing
    every shift.  Returns (r, groups) in the rotation-sum conventions."""
    a = map_slots(C, H, W, *src)
    b = map_slots(C, H, W, *dst)
    diags = {}
    for s_, d_ in zip(a, b):
        o = int((s_ - d_) % nslots)
        diags.setdefault(o, np.zeros(nslots))[int(d_)] = 1.0
    stride = nslots
    for o in diags:
        while stride > 1 and o % stride:
            stride //= 2
    return bsgs_plan(diags, nslots, stride)


def resnet_fp64(X, w, chans, nblocks, betas=None, D=RELU_DEGREE, perturb=None):
    """ResNet-20-style network (paper's Appendix A architecture) in FP64 from the
    plain layers: 3x3 conv + ReLU; per stage, residual blocks (3x3 conv, ReLU,
    3x3 conv, + shortcut, ReLU) whose first block in stages 2 and 3 has stride
    2 and a 1x1 stride-2 conv shortcut; global average pooling; FC.  With
    `betas`, ReLU i is the Chebyshev series of Alg. 4 with bound betas[i].
    perturb(i, v), when given, returns the input ReLU i then takes (an error
    model: what an encrypted pipeline adds before that ReLU)."""
    idx = [0]

    def act(v):
        i = idx[0]
        idx[0] += 1
        if perturb is not None:
            v = perturb(i, v)
        return np.maximum(v, 0.0) if betas is None else relu_fp64(v, betas[i], D)

    h = act(conv2d_fp64(X, w["conv0"][0], b=w["conv0"][1], pad=1))
    for s in range(len(chans)):
        for bk in range(nblocks):
            name = "s%db%d" % (s, bk)
            st = 2 if (s > 0 and bk == 0) else 1
            t = act(conv2d_fp64(h, w[name + "_a"][0], b=w[name + "_a"][1], stride=st, pad=1))
            t = conv2d_fp64(t, w[name + "_b"][0], b=w[name + "_b"][1], pad=1)
            sc = conv2d_fp64(h, w[name + "_sc"][0], b=w[name + "_sc"][1], stride=2) if st == 2 else h
            h = act(t + sc)
    g = avgpool_fp64(h, h.shape[1], h.shape[1]).reshape(-1)
    Wf, bf = w["fc"]
    return Wf @ g + bf
