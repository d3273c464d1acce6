"""FHEON's own layer algorithms, step by step on FP64 slot vectors, with the
rotations, keys, plaintext products and depth each one spends.

TEST INFRASTRUCTURE: only the tests may import this module.

The library does not run these forms: its layers are rotation-sum plans
(oracle/fheon.py restates those).  This module restates what the paper's
Sec. 5.1 (convolution with the A* mask and output extraction), Sec. 5.2
(padding by rotations; striding by extraction, approach 1; striding by masks,
approach 2, also over several channels at once), Sec. 5.4 (average and
global average pooling) and Sec. 5.5 (fully connected layer with merge
rotations) compute, so that the tests can pin them against the plain layer
equations and the paper's own key and rotation counts, and show that the
library's plans give the same values.

Layout: the paper's flattened tensor, channel c of a (C, H, W) map in the
block at c*H*W, position (h, w) at c*H*W + h*W + w (Sec. 5.1, input
flattening).  Rot_r moves slot i+r to slot i (r > 0 rotates left), as in
Algorithm 1.  Where the paper's text leaves a step open, the reading taken
is stated at the function.
"""
import math

import numpy as np


class Ct:
    """A slot vector standing for a ciphertext, with the number of plaintext
    products on its longest path (its multiplicative depth)."""

    def __init__(self, v, depth=0):
        self.v = np.asarray(v, dtype=np.float64)
        self.depth = depth


class Counter:
    """Records every rotation amount and plaintext product of a pipeline."""

    def __init__(self, nslots):
        self.n = nslots
        self.rotations = []
        self.products = 0

    def rot(self, x, r):
        if r % self.n == 0:
            return x
        self.rotations.append(int(r))
        return Ct(np.roll(x.v, -r), x.depth)

    def mul(self, x, p):
        self.products += 1
        return Ct(x.v * np.asarray(p, dtype=np.float64), x.depth + 1)

    @staticmethod
    def add(a, b):
        if a is None:
            return b
        return Ct(a.v + b.v, max(a.depth, b.depth))

    def add_plain(self, x, p):
        return Ct(x.v + np.asarray(p, dtype=np.float64), x.depth)

    @property
    def keys(self):
        """The distinct rotation amounts: one rotation key each."""
        return set(self.rotations)


def flatten(X, nslots):
    """A (C, H, W) tensor at slots c*H*W + h*W + w, zero elsewhere."""
    v = np.zeros(nslots)
    X = np.asarray(X, dtype=np.float64)
    v[:X.size] = X.reshape(-1)
    return v


def unflatten(v, shape):
    return np.asarray(v)[:int(np.prod(shape))].reshape(shape)


def ones_at(n, slots):
    m = np.zeros(n)
    m[np.asarray(list(slots), dtype=np.int64)] = 1.0
    return m


# ------------------------------------------------------------------ Sec. 5.1
def conv_astar(cnt, x, C, H, W, K, f, taps=None):
    """Sec. 5.1, first part, for output channel f of a C-channel H x W map:
    the k^2 - 1 rotations Rot_{i*W + j}(x) (made once for every output
    channel; pass them in `taps`), each times its repeated kernel vector (in
    channel c's block the value K[f, c, i, j]), summed into A; A, Rot_{W^2}(A),
    Rot_{W^2}(Rot_{W^2}(A)), ... (C of them, each rotation by the one W^2 key
    applied to the previous one) summed, which brings every channel's partial
    sum to block 0; then the A* mask, read as W^2 ones followed by
    (C - 1) W^2 zeros (H*W for a non-square map).  Returns (A*, taps): A*
    holds the stride-1 valid-convolution value of output (h, w) at h*W + w."""
    n = cnt.n
    k = K.shape[2]
    B = H * W
    if taps is None:
        taps = {(i, j): cnt.rot(x, i * W + j) for i in range(k) for j in range(k)}
    A = None
    for i in range(k):
        for j in range(k):
            kv = np.zeros(n)
            for c in range(C):
                kv[c * B:(c + 1) * B] = K[f, c, i, j]
            A = cnt.add(A, cnt.mul(taps[(i, j)], kv))
    S, cur = A, A
    for _ in range(1, C):
        cur = cnt.rot(cur, B)
        S = cnt.add(S, cur)
    Astar = cnt.mul(S, ones_at(n, range(B))) if C > 1 else S
    return Astar, taps


def extract_rows(cnt, Astar, Wa, Ho, Wo):
    """Sec. 5.1, output extraction (stride 1): row i of A* (slots i*Wa ..)
    goes to i*Wo.  T_0 = A*, T_i = Rot_{Wa - Wo}(T_{i-1}) puts row i at i*Wo;
    one row mask per output row keeps it.  Reading: the printed 'single
    rotation key of W_out' is read as the key of Wa - Wo (= k - 1 without
    padding, itself the tap key Rot_{k-1}), the shift between consecutive rows
    of A* and of the output."""
    n = cnt.n
    y, T = None, Astar
    for i in range(Ho):
        if i > 0:
            T = cnt.rot(T, Wa - Wo)
        y = cnt.add(y, cnt.mul(T, ones_at(n, range(i * Wo, (i + 1) * Wo))))
    return y


def place_channels(cnt, ys, block):
    """Sec. 5.1: output channel f moved to block f by Rot_{-f * block} (one
    key per output channel f >= 1), all added into one ciphertext."""
    y = None
    for f, yf in enumerate(ys):
        y = cnt.add(y, cnt.rot(yf, -f * block))
    return y


def bias_vector(n, b, F, block, count):
    v = np.zeros(n)
    for f in range(F):
        v[f * block:f * block + count] = b[f]
    return v


def conv(cnt, x, C, H, W, K, b=None):
    """Sec. 5.1 convolution (no padding, stride 1) of a C x H x W map with a
    (F, C, k, k) kernel: A* per output channel (conv_astar), its extraction
    (extract_rows), channel placement at f * Ho * Wo, bias.  Output: the
    flattened (F, Ho, Wo) map, Ho = H - k + 1, Wo = W - k + 1."""
    F, _, k, _ = K.shape
    Ho, Wo = H - k + 1, W - k + 1
    ys, taps = [], None
    for f in range(F):
        Astar, taps = conv_astar(cnt, x, C, H, W, K, f, taps)
        ys.append(extract_rows(cnt, Astar, W, Ho, Wo))
    y = place_channels(cnt, ys, Ho * Wo)
    if b is not None:
        y = cnt.add_plain(y, bias_vector(cnt.n, b, F, Ho * Wo, Ho * Wo))
    return y


# ------------------------------------------------------------------ Sec. 5.2 padding
def pad(cnt, x, C, H, W, P):
    """Sec. 5.2 padding by rotations: (C, H, W) -> flattened (C, H+2P, W+2P).
    Per channel c, its rows (one mask each) are joined from the last row up,
    acc = Rot_{-2P}(acc) + row_h: the one rotation between two sequential
    rows opens the 2P zeros of the row ends (H - 1 rotations, key -2P).  One
    more rotation, by -(c (Hp Wp - H W) + P Wp + P), puts the channel at its
    padded block and opens the leading zeros (P Wp + P; the printed W_p + P
    is that count at P = 1).  H rotations per channel (W for square maps);
    C + 1 keys.  Reading: the paper's separate channel move by W^2 and its
    leading-zero shift are the one placement rotation here, so its C + 3 keys
    are an upper bound."""
    n = cnt.n
    Hp, Wp = H + 2 * P, W + 2 * P
    y = None
    for c in range(C):
        acc = None
        for h in range(H - 1, -1, -1):
            row = cnt.mul(x, ones_at(n, range(c * H * W + h * W, c * H * W + (h + 1) * W)))
            acc = row if acc is None else cnt.add(cnt.rot(acc, -2 * P), row)
        y = cnt.add(y, cnt.rot(acc, -(c * (Hp * Wp - H * W) + P * Wp + P)))
    return y


# ------------------------------------------------------------------ Sec. 5.2 striding
def stride_extract(cnt, Astar, Wa, Ho, Wo, S):
    """Sec. 5.2 striding, approach 1, on A* (stride-1 results at r*Wa + s):
    output (i, j) is A* at (S i, S j).  Vertical: T_0 = A*, T_i =
    Rot_{S Wa}(T_{i-1}) brings row S i to slot 0.  Horizontal: value S j of
    T_i moves to j by Rot_{(S-1) j} and is kept by a one-slot mask; the Wo
    values of a row are summed.  Rows are joined from the last one up by
    acc = Rot_{-Wo}(acc) + row_i.  Keys: S Wa, (S-1) j for 1 <= j < Wo, -Wo:
    Wo + 1 (the paper counts Wo + 2).  Output: (Ho, Wo) flattened."""
    n = cnt.n
    rows, T = [], Astar
    for i in range(Ho):
        if i > 0:
            T = cnt.rot(T, S * Wa)
        r = None
        for j in range(Wo):
            r = cnt.add(r, cnt.mul(cnt.rot(T, (S - 1) * j), ones_at(n, [j])))
        rows.append(r)
    acc = rows[-1]
    for i in range(Ho - 2, -1, -1):
        acc = cnt.add(cnt.rot(acc, -Wo), rows[i])
    return acc


def stride_masks(cnt, x, Wa, Ba, Ho, Wo, S, g=1):
    """Sec. 5.2 striding, approach 2, on g maps at once (the multi-channel
    pipeline: channel f's stride-1 results at f*Ba + r*Wa + s):
      1. one mask keeps the stride-aligned values (S i, S j), i < Ho, j < Wo;
      2. ceil(log2 Wo) steps compact the columns: at step t the values whose
         output column j has bit t set move left by (S-1) 2^t (a mask on the
         movers, a rotation, a mask on the rest, summed), so column S j ends
         at j;
      3. the rows: U_0 = x, U_i = Rot_{S Wa - Wo}(U_{i-1}) puts row i of every
         channel at i*Wo, and one mask per output row keeps it; for g > 1 the
         channels first step by Rot_{Ba - Ho Wo} (V_f = Rot(V_{f-1})), so that
         row i of channel f lands at (f Ho + i) Wo.
    Keys: ceil(log2 Wo) + 1 (+1 for g > 1: the channel step); rotations
    ceil(log2 Wo) + Ho - 1 for one channel.  Output: (g, Ho, Wo) flattened."""
    n = cnt.n
    steps = max(0, math.ceil(math.log2(Wo))) if Wo > 1 else 0
    pos = {(f, i, j): f * Ba + S * i * Wa + S * j for f in range(g) for i in range(Ho) for j in range(Wo)}
    y = cnt.mul(x, ones_at(n, pos.values()))
    for t in range(steps):
        d = (S - 1) << t
        mv = [key for key in pos if (key[2] >> t) & 1]
        st = [key for key in pos if not (key[2] >> t) & 1]
        moved = cnt.rot(cnt.mul(y, ones_at(n, [pos[key] for key in mv])), d)
        kept = cnt.mul(y, ones_at(n, [pos[key] for key in st]))
        y = cnt.add(kept, moved)
        for key in mv:
            pos[key] -= d
    # every value now sits at f*Ba + S*i*Wa + j
    out, V = None, y
    for f in range(g):
        if f > 0:
            V = cnt.rot(V, Ba - Ho * Wo)
        U = V
        for i in range(Ho):
            if i > 0:
                U = cnt.rot(U, S * Wa - Wo)
            base = (f * Ho + i) * Wo
            out = cnt.add(out, cnt.mul(U, ones_at(n, range(base, base + Wo))))
    return out


def conv_advanced(cnt, x, C, H, W, K, b=None, P=0, S=1, approach=2, joint=False):
    """Sec. 5.2 convolution with padding P and stride S: padding by rotations
    (pad), then A* of every output channel on the padded map (conv_astar),
    then the output positions: S = 1 by the row extraction of Sec. 5.1, S > 1
    by striding approach 1 (stride_extract) or 2 (stride_masks, per channel;
    joint=True: the A* of all F channels concatenated at blocks of Hp Wp and
    strided at once), then channel placement and bias.  Output: flattened
    (F, Ho, Wo), Ho = (H + 2P - k)/S + 1."""
    F, _, k, _ = K.shape
    Hp, Wp = H + 2 * P, W + 2 * P
    Ho, Wo = (Hp - k) // S + 1, (Wp - k) // S + 1
    xp = pad(cnt, x, C, H, W, P) if P else x
    stars, taps = [], None
    for f in range(F):
        Astar, taps = conv_astar(cnt, xp, C, Hp, Wp, K, f, taps)
        stars.append(Astar)
    if S > 1 and approach == 2 and joint:
        cat = place_channels(cnt, stars, Hp * Wp)
        y = stride_masks(cnt, cat, Wp, Hp * Wp, Ho, Wo, S, g=F)
    else:
        ys = []
        for A in stars:
            if S == 1:
                ys.append(extract_rows(cnt, A, Wp, Ho, Wo))
            elif approach == 1:
                ys.append(stride_extract(cnt, A, Wp, Ho, Wo, S))
            else:
                ys.append(stride_masks(cnt, A, Wp, Hp * Wp, Ho, Wo, S))
        y = place_channels(cnt, ys, Ho * Wo)
    if b is not None:
        y = cnt.add_plain(y, bias_vector(cnt.n, b, F, Ho * Wo, Ho * Wo))
    return y


# ------------------------------------------------------------------ Sec. 5.4
def avgpool(cnt, x, C, H, W, k, S, approach=2):
    """Sec. 5.4 average pooling: the window sum by the convolution's
    rotations Rot_{i W + j}(x) (i, j < k), summed and times the repeated
    1/k^2, then the striding of Sec. 5.2 over all C channels (approach 2 with
    the multi-channel pipeline, or approach 1 per channel followed by the
    channel placement).  Output: flattened (C, Ho, Wo), Ho = (H - k)/S + 1."""
    n = cnt.n
    Ho, Wo = (H - k) // S + 1, (W - k) // S + 1
    A = None
    for i in range(k):
        for j in range(k):
            A = cnt.add(A, cnt.rot(x, i * W + j))
    A = cnt.mul(A, np.full(n, 1.0 / (k * k)))
    if approach == 2:
        return stride_masks(cnt, A, W, H * W, Ho, Wo, S, g=C)
    ys = []
    for c in range(C):
        ys.append(stride_extract(cnt, cnt.rot(A, c * H * W), W, Ho, Wo, S))
    return place_channels(cnt, ys, Ho * Wo)


def global_avgpool(cnt, x, C, H, W):
    """Sec. 5.4 global average pooling: the sum of each channel's H*W values
    by rotate-and-add (steps 1, 2, 4, ..., below H*W, so slot c*H*W holds
    channel c's sum when H*W is a power of two), then each channel's first
    value merged into slot c by one key (V_c = Rot_{H W - 1}(V_{c-1})), with
    the one-slot mask carrying 1/(H W).  Output: the C means in slots 0..C-1."""
    n = cnt.n
    B = H * W
    assert B & (B - 1) == 0, "the rotate-and-add sum needs H*W a power of two"
    s = x
    st = 1
    while st < B:
        s = cnt.add(s, cnt.rot(s, st))
        st *= 2
    y, V = None, s
    for c in range(C):
        if c > 0:
            V = cnt.rot(V, B - 1)
        e = np.zeros(n)
        e[c] = 1.0 / B
        y = cnt.add(y, cnt.mul(V, e))
    return y


# ------------------------------------------------------------------ Sec. 5.5
def fc(cnt, x, Wmat, b, in_slots, max_keys=None):
    """Sec. 5.5 fully connected layer: per output neuron k, one product by its
    weights at the input's slots and the sum of the slots by rotate-and-add
    (log2 n rotations by powers of two; the paper's 'n additions'), which
    leaves the total in every slot; then the merge of the m totals into slots
    0..m-1.  Merge, with a budget of max_keys keys (the paper's parameter):
    at least m - 1 keys: neuron k's slot 0 (one-slot mask) moved by Rot_{-k};
    fewer: blocks of B = ceil(m / max_keys) neurons, each joined from its last
    neuron down by acc = Rot_{-1}(acc) + e_0 t_k, then moved to its first
    slot by Rot_{-start} (max_keys keys at most, for max_keys >= 1)."""
    n = cnt.n
    Wmat = np.asarray(Wmat, dtype=np.float64)
    m = Wmat.shape[0]
    ts = []
    for kk in range(m):
        w = np.zeros(n)
        w[np.asarray(in_slots)] = Wmat[kk]
        t = cnt.mul(x, w)
        st = 1
        while st < n:
            t = cnt.add(t, cnt.rot(t, st))
            st *= 2
        ts.append(t)
    e0 = ones_at(n, [0])
    if max_keys is None or max_keys >= m - 1:
        y = None
        for kk, t in enumerate(ts):
            y = cnt.add(y, cnt.rot(cnt.mul(t, e0), -kk))
    else:
        assert max_keys >= 1
        B = -(-m // max_keys)
        y = None
        for start in range(0, m, B):
            blk = list(range(start, min(m, start + B)))
            acc = cnt.mul(ts[blk[-1]], e0)
            for kk in reversed(blk[:-1]):
                acc = cnt.add(cnt.rot(acc, -1), cnt.mul(ts[kk], e0))
            y = cnt.add(y, cnt.rot(acc, -start))
    if b is not None:
        bv = np.zeros(n)
        bv[:m] = b
        y = cnt.add_plain(y, bv)
    return y
