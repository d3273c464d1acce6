"""CKKS bootstrapping, restated for the oracle.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

The paper offers bootstrapping as a layer that can be placed anywhere in a
network ("Bootstrapping Layer" among the support functions; in the evaluation
it runs before every ReLU but the first two, before the second pooling layer
and before the global pooling) and takes the algorithm from its library.  The
steps here are the published full-slot bootstrapping of Cheon, Han, Kim, Kim
and Song (Eurocrypt 2018), with the linear transforms factored into the
butterfly stages of the special FFT and evaluated in baby-step/giant-step form
(Chen, Chillotti and Song, Eurocrypt 2019) and the modular reduction as a
scaled cosine followed by double-angle steps (Han and Ki, CT-RSA 2020):

  1. ModRaise: the input at level 1 (modulus q_0) is taken to coefficient
     form, lifted to centred integers and reduced into every prime of Q.  It
     now decrypts to t = m + q_0 I with I a small integer polynomial.
  2. CoeffToSlot: slots hold w = F (t_lo + i t_hi) (F: evaluation at the slot
     roots of a degree < N/2 polynomial, t_lo / t_hi the low / high half of
     the coefficients).  The inverse butterfly stages of F, merged into
     `cts_levels` groups, each one BSGS linear layer, give
     (t_lo + i t_hi) / (2 K q_0) in bit-reversed slot order.
  3. Real and imaginary parts: with the conjugate c' (Galois element 2N - 1),
     c + c' holds t_lo / (K q_0) and i (c' - c) holds t_hi / (K q_0).
  4. EvalMod, on each part x = t / (K q_0) in [-1, 1]: the Chebyshev series of
     cos(2 pi (K x - 1/4) / 2^r), then r steps c <- 2 c^2 - 1, which give
     sin(2 pi t / q_0) = sin(2 pi m / q_0) ~= 2 pi m / q_0.
  5. Recombination: re + i im.
  6. SlotToCoeff: the butterfly stages of F, merged into `stc_levels` groups,
     with the factor q_0 / (2 pi Delta) folded into the first, give back the
     slots of m / Delta = the input's message.

Sparse bootstrap (a message in slots [0, ns), ns <= N/4; the library the
paper runs does the same for fewer than N/2 slots): with copies = N / (2 ns),
  0. the input (level >= 2) times the mask of slots [0, ns), rescaled, then
     repeated in every copy of ns slots by x += Rot_{ns 2^j}(x): its
     polynomial now lies in Z[X^copies];
  1. ModRaise as above, then the trace x += Rot_{ns 2^j}(x), which keeps
     copies times the coefficients of X^(copies k) of t and drops the rest;
  2. CoeffToSlot: the ns-slot transform of that subring in every copy (its
     slots are the ns-slot ring's slots of T(Y) = t(X), Y = X^copies),
     1 / copies folded into the first level and the copy factor (1 on even
     copies, -i on odd ones) into the last, so that y + conj(y) holds
     T_lo / (K q_0) in the even copies and T_hi / (K q_0) in the odd ones;
  3. ONE EvalMod on y + conj(y);
  4. SlotToCoeff: the map (a, b) -> a + i b in every copy (diagonals
     {0: (1, i), ns: (i, 1)}), composed into the first level, then the
     ns-slot transform in every copy.
The output holds the input's slots [0, ns) in every copy.

Slot convention: slot j is the evaluation at zeta^(5^j mod 2N), zeta =
exp(i pi / N); Rot_k moves slot j + k to slot j.
"""
import ctypes
import math

import numpy as np

from . import ckks
from . import fheon as OF


# ------------------------------------------------------------------ the special FFT
def brv(x, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


def stage_diagonals(n, h, inverse=False):
    """Butterfly stage of half-length h of F (or its inverse) as slot diagonals
    {offset mod n: complex vector}: out = sum_o d_o * Rot_o(in).

    Stage h (blocks of m = 2h slots, u = position in the block, u < h):
      out[b+u]   = in[b+u] + w_u in[b+u+h]
      out[b+u+h] = in[b+u] - w_u in[b+u+h],   w_u = exp(2 pi i (5^u mod 4m) / 4m).
    Its inverse: in[b+u] = (out[b+u] + out[b+u+h]) / 2,
                 in[b+u+h] = (out[b+u] - out[b+u+h]) / (2 w_u)."""
    m = 2 * h
    j = np.arange(n)
    u = j % m
    lo = u < h
    uu = np.where(lo, u, u - h)
    e = np.array([pow(5, int(x), 4 * m) for x in uu], dtype=np.float64)
    w = np.exp(2j * np.pi * e / (4 * m))
    if not inverse:
        d0 = np.where(lo, 1.0 + 0j, -w)
        dp = np.where(lo, w, 0j)
        dm = np.where(lo, 0j, 1.0 + 0j)
    else:
        d0 = np.where(lo, 0.5 + 0j, -0.5 / w)
        dp = np.where(lo, 0.5 + 0j, 0j)
        dm = np.where(lo, 0j, 0.5 / w)
    out = {}
    for o, d in ((0, d0), (h % n, dp), ((-h) % n, dm)):
        out[o] = out.get(o, 0j) + d
    return out


def apply_diagonals(diags, v):
    """sum_o d_o * Rot_o(v) in FP64."""
    out = np.zeros(len(v), dtype=np.complex128)
    for o, d in diags.items():
        out += d * np.roll(v, -o)
    return out


def compose(A, B, n):
    """Diagonals of A.B (B applied first): (A B v)[j] = sum_a A_a[j] (B v)[j + a]."""
    C = {}
    for a, da in A.items():
        for b, db in B.items():
            c = (a + b) % n
            C[c] = C.get(c, 0j) + da * np.roll(db, -a)
    return C


def stage_groups(logn, levels):
    """Stages 1..logn (stage s has half-length 2^(s-1)) split into `levels`
    consecutive groups, the larger groups at the top."""
    base, extra = divmod(logn, levels)
    sizes = [base + (1 if g >= levels - extra else 0) for g in range(levels)]
    groups, s = [], 1
    for sz in sizes:
        groups.append(list(range(s, s + sz)))
        s += sz
    return groups


def stc_levels(n, levels):
    """Merged SlotToCoeff groups in the order they are applied (low stages
    first): each the product of its stages' diagonals."""
    logn = n.bit_length() - 1
    out = []
    for g in stage_groups(logn, levels):
        M = None
        for s in g:
            S = stage_diagonals(n, 1 << (s - 1))
            M = S if M is None else compose(S, M, n)
        out.append((1 << (g[0] - 1), M))
    return out


def replicate(M, ns, n):
    """Diagonals of an ns-slot map as an n-slot map for inputs of period ns
    (ns divides n): every vector tiled n/ns times, offset o in [0, ns) taken
    as o or o - ns, whichever is nearer to 0, modulo n.  On an input whose
    slots repeat every ns it computes the ns-slot map in every copy."""
    out = {}
    for o, d in M.items():
        oo = (o if o <= ns // 2 else o - ns) % n
        out[oo] = out.get(oo, 0j) + np.tile(d, n // ns)
    return out


def copy_factor(ns, n):
    """1 on the even copies of ns slots, -i on the odd ones.  CoeffToSlot of a
    sparse bootstrap ends with it: with y = f * u (u repeated), y + conj(y)
    holds 2 Re u in the even copies and 2 Im u in the odd ones."""
    return np.tile(np.concatenate([np.ones(ns), np.full(ns, -1j)]), n // (2 * ns))


def join_map(ns, n):
    """Diagonals {0: P1, ns: P2} of the map from w = (a, b) (period 2 ns, real
    a and b) to a + i b repeated every ns slots: P1 = (1, i), P2 = (i, 1), so
    that copy 2c gets a + i b and copy 2c + 1 gets i b + a."""
    one, im = np.ones(ns), np.full(ns, 1j)
    return {0: np.tile(np.concatenate([one, im]), n // (2 * ns)),
            ns % n: np.tile(np.concatenate([im, one]), n // (2 * ns))}


def cts_levels(n, levels):
    """Merged CoeffToSlot groups in the order they are applied (top stages
    first): each the product of its stages' inverse diagonals."""
    logn = n.bit_length() - 1
    out = []
    for g in reversed(stage_groups(logn, levels)):
        M = None
        for s in reversed(g):
            S = stage_diagonals(n, 1 << (s - 1), inverse=True)
            M = S if M is None else compose(S, M, n)
        out.append((1 << (g[0] - 1), M))
    return out


def cts_levels_sparse(n, ns, levels):
    """CoeffToSlot of the sparse bootstrap on n slots: the ns-slot levels in
    every copy (replicate), the last one times the copy factor (1, -i)."""
    out = [(stride, replicate(M, ns, n)) for stride, M in cts_levels(ns, levels)]
    stride, M = out[-1]
    f = copy_factor(ns, n)
    out[-1] = (stride, {o: d * f for o, d in M.items()})
    return out


def stc_levels_sparse(n, ns, levels):
    """SlotToCoeff of the sparse bootstrap on n slots: the join map from
    (a, b) to a + i b, then the ns-slot levels in every copy."""
    out = [(stride, replicate(M, ns, n)) for stride, M in stc_levels(ns, levels)]
    _, M = out[0]
    out[0] = (1, compose(M, join_map(ns, n), n))
    return out


# BSGS plans of the merged levels (shared with the repacking layer)
bsgs_plan = OF.bsgs_plan
plan_slots = OF.plan_slots


# ------------------------------------------------------------------ parameters
def default_K(N):
    """Bound K on |t / q_0| for a uniform ternary secret: a coefficient of
    c_1 s sums about 2N/3 terms uniform in [-q_0/2, q_0/2), so t / q_0 has
    standard deviation about sqrt(N / 18); K is the power of two at or above
    8 of those."""
    x = 8.0 * math.sqrt(N / 18.0)
    K = 1
    while K < x:
        K *= 2
    return K


def default_doublings(K):
    """r with 2^r >= K: the cosine's argument spans at most one period."""
    r = 0
    while (1 << r) < K:
        r += 1
    return r


BOOT_DEGREE = 27


def evalmod_coeffs(K, r, D=BOOT_DEGREE):
    """Chebyshev coefficients of cos(2 pi (K z - 1/4) / 2^r) on [-1, 1] (C oracle)."""
    from . import _lib
    out = (ctypes.c_double * (D + 1))()
    _lib.lib().oracle_cos_cheb_coeffs(float(K), int(r), int(D), out)
    return np.array(out[:], dtype=np.float64)


def evalmod_fp64(x, K, r, D=BOOT_DEGREE):
    """FP64 value of EvalMod on x in [-1, 1]: the series, then r doublings."""
    c = OF.cheb_eval_fp64(evalmod_coeffs(K, r, D), x)
    for _ in range(r):
        c = 2.0 * c * c - 1.0
    return c


def depth(cts, stc, D, r):
    """Levels a bootstrap consumes."""
    return cts + OF.cheb_depth(D) + r + stc


class Plan:
    """Everything the bootstrap of one context needs besides the keys: the
    merged CoeffToSlot and SlotToCoeff levels as BSGS plans (complex FP64
    vectors), their plaintexts' scales, EvalMod's coefficients.

    Scales: the raised ciphertext carries scale q_0 (its slots are F(t)/q_0).
    CoeffToSlot's first level folds 1 / (2K) into its vectors and encodes them
    at q_{l-1} * (Delta_b / q_0), Delta_b = the prime EvalMod's first product
    is rescaled by; the others at q_{l-1}.  SlotToCoeff's first level folds
    q_0 / (2 pi Delta_in) into its vectors; its last level is encoded at
    q_{l-1} * (Delta_in / S) (S: the scale before it), the others at q_{l-1}:
    all but the last level run at EvalMod's scale, where key-switching noise
    is small against the message.  The output then has scale ~= Delta_in and
    the input's message."""

    def __init__(self, ctx, in_scale, cts=3, stc=3, K=None, r=None, D=BOOT_DEGREE, baby=0, slots=None,
                 masked=True):
        N, L = ctx.N, ctx.L
        n = N // 2
        ns = n if not slots else int(slots)
        if ns > n or ns < 2 or ns & (ns - 1):
            raise ValueError("slots: a power of two in [2, N/2]")
        self.N, self.n, self.in_scale = N, n, float(in_scale)
        # sparse (ns < N/2): the message lives in slots [0, ns); copies = n / ns;
        # unmasked (masked=False): the inputs are zero outside those slots
        self.ns, self.copies = ns, n // ns
        self.masked = bool(masked) or ns == n
        self.K = K or default_K(N)
        self.r = default_doublings(self.K) if r is None else r
        self.D, self.ncts, self.nstc = D, cts, stc
        self.coeffs = evalmod_coeffs(self.K, self.r, D)
        q = [float(x) for x in ctx.q]
        if depth(cts, stc, D, self.r) > L - 1:
            raise ValueError("bootstrap needs %d levels above q_0" % depth(cts, stc, D, self.r))
        lv = L
        # CoeffToSlot (sparse: the ns-slot transform in every copy, after the
        # trace summed the copies, which multiplied the message by `copies`)
        self.cts = []
        s = float(ctx.q[0])
        delta_b = q[L - cts - 1]
        for i, (stride, M) in enumerate(cts_levels(n, cts) if ns == n else cts_levels_sparse(n, ns, cts)):
            if i == 0:
                M = {o: d * (1.0 / (2.0 * self.K * self.copies)) for o, d in M.items()}
                ps = q[lv - 1] * (delta_b / float(ctx.q[0]))
            else:
                ps = q[lv - 1]
            rr, groups = bsgs_plan(M, n, stride, baby)
            self.cts.append((rr, groups, ps, lv))
            s = (s * ps) / q[lv - 1]
            lv -= 1
        self.cts_scale = s
        # EvalMod: the series keeps the scale; each doubling squares it and rescales
        lv -= OF.cheb_depth(D)
        for _ in range(self.r):
            s = (s * s) / q[lv - 1]
            lv -= 1
        self.evalmod_scale = s
        # SlotToCoeff (sparse: the first level starts with the join map from
        # the real parts (a, b) to a + i b in every copy)
        self.stc = []
        for i, (stride, M) in enumerate(stc_levels(n, stc) if ns == n else stc_levels_sparse(n, ns, stc)):
            if i == 0:
                M = {o: d * (float(ctx.q[0]) / (2.0 * math.pi * self.in_scale)) for o, d in M.items()}
            ps = q[lv - 1] * (self.in_scale / s) if i == stc - 1 else q[lv - 1]
            rr, groups = bsgs_plan(M, n, stride, baby)
            self.stc.append((rr, groups, ps, lv))
            s = (s * ps) / q[lv - 1]
            lv -= 1
        self.out_scale, self.out_level = s, lv

    def trace_steps(self):
        """Rotation steps of the trace over the copies (ns, 2 ns, ...): sparse only."""
        return [self.ns << j for j in range(self.copies.bit_length() - 1)]

    def mask_slots(self):
        """The sparse bootstrap's input mask: 1 in slots [0, ns), 0 elsewhere."""
        v = np.zeros(self.n)
        v[:self.ns] = 1.0
        return v

    def steps(self):
        """Rotation steps of the plan's keys (besides the conjugation)."""
        st = set(self.trace_steps()) if self.ns < self.n else set()
        for rr, groups, _, _ in self.cts + self.stc:
            st |= set(OF.linear_steps(rr, groups))
        return sorted(st)

    def encode(self, ctx):
        """Plaintexts of every level: [[per group, per tap: u64[level][N] or None]]."""
        out = []
        for rr, groups, ps, lv in self.cts + self.stc:
            out.append([[None if v is None else ctx.plain_from_coeffs(ckks.encode(v, self.N, ps), lv)
                         for v in vals] for _, vals in groups])
        return out

    def encode_mask(self, ctx):
        """The sparse input mask as a plaintext at level 2, scale q_1 (the
        prime its rescale drops, so the scale is kept)."""
        return ctx.plain_from_coeffs(ckks.encode(self.mask_slots(), self.N, float(ctx.q[1])), 2)


def mod_raise(ctx, ct):
    """A level-1 ciphertext (modulus q_0) raised to all L primes: each component
    to coefficients mod q_0, centred (values above q_0 // 2 less q_0), reduced
    into every q_i, back to the evaluation domain."""
    q0 = int(ctx.q[0])
    out = np.zeros((2, ctx.L, ctx.N), dtype=np.uint64)
    for b in range(2):
        c = ctx.to_coeff(np.ascontiguousarray(ct[b, :1]), 1)[0].astype(np.int64)
        c = np.where(c > q0 // 2, c - q0, c)
        res = np.stack([(c % int(qi)).astype(np.uint64) for qi in ctx.q])
        out[b] = ctx.to_eval(res, ctx.L)
    return out


def monomial(ctx, level, sign=1):
    """sign * X^(N/2) as a plaintext (the constant sign * i in every slot, scale 1)."""
    m = np.zeros(ctx.N, dtype=np.int64)
    m[ctx.N // 2] = sign
    return ctx.plain_from_coeffs(m, level)


def double_angle(ctx, c, scale, rlk):
    """2 c^2 - 1: the doubled product rescaled, then -1 at the new scale."""
    lv = c.shape[1]
    prod = ctx.mul_relin(ctx.mul_int(c, 2), c, rlk)
    sc = (scale * scale) / float(ctx.q[lv - 1])
    return ctx.add_const(ctx.rescale(prod), -1.0, sc), sc


def bootstrap_encrypted(ctx, ct, plan, pts, keys, rlk, conj_key, trace=None, mask=None):
    """The six steps on a ciphertext of scale plan.in_scale at any level >= 1
    (returns (ct, scale)).  pts: plan.encode(ctx); keys: step -> key;
    trace (optional dict) receives the intermediate ciphertexts.

    Sparse plans (plan.ns < N/2; the input at level >= 2, mask =
    plan.encode_mask(ctx); unmasked plans: inputs zero outside slots [0, ns),
    at level >= 1, no mask) take the message of slots [0, ns) only and
    return it in every copy of ns slots: the input is masked to those slots
    and repeated in every copy (so its polynomial lies in Z[X^copies]);
    after ModRaise the trace (the sum of the copies' rotations) removes the
    other coefficients of q_0 I; CoeffToSlot is the ns-slot transform of
    that subring, ending in the copy factor (1, -i); one EvalMod runs on
    y + conj(y) = (T_lo, T_hi) / (K q_0); SlotToCoeff starts with the join
    map back to T_lo + i T_hi in every copy."""
    N = ctx.N
    sparse = plan.ns < plan.n
    if sparse:
        # slots [0, ns) kept, repeated in every copy: the message then lies in
        # the subring the trace below projects onto (an unmasked plan's inputs
        # are zero outside those slots already)
        if plan.masked:
            x = ctx.rescale(ctx.mul_plain(ctx.drop_level(ct, 2), mask))
        else:
            x = ctx.drop_level(ct, 1)
        for st in plan.trace_steps():
            x = ctx.add(x, ctx.rotate(x, ckks.galois_elt(st, N), keys[st]))
        if trace is not None:
            trace["repeated"] = x
        x = mod_raise(ctx, x)
    else:
        x = mod_raise(ctx, ctx.drop_level(ct, 1))
    if trace is not None:
        trace["raised"] = x
    if sparse:
        # the trace: the sum of the copies' automorphisms, which keeps the
        # coefficients of X^(copies j) (times copies) and drops the others
        for st in plan.trace_steps():
            x = ctx.add(x, ctx.rotate(x, ckks.galois_elt(st, N), keys[st]))
        if trace is not None:
            trace["traced"] = x
    s = float(ctx.q[0])
    levels = plan.cts + plan.stc
    for i, (rr, groups, ps, lv) in enumerate(plan.cts):
        x = OF.linear_encrypted(ctx, x, rr, groups, pts[i], keys)
        s = (s * ps) / float(ctx.q[lv - 1])
    if trace is not None:
        trace["cts"] = x
    xc = ctx.rotate(x, 2 * N - 1, conj_key)
    lv = x.shape[1]
    if sparse:
        # one part: 2 Re u in the even copies, 2 Im u in the odd ones
        c = OF.cheb_encrypted(ctx, ctx.add(x, xc), s, plan.coeffs, rlk)
        sc = s
        for _ in range(plan.r):
            c, sc = double_angle(ctx, c, sc, rlk)
        s = sc
        if trace is not None:
            trace["evalmod"] = [c]
        y = c
        for i, (rr, groups, ps, lv) in enumerate(plan.stc):
            y = OF.linear_encrypted(ctx, y, rr, groups, pts[len(plan.cts) + i], keys)
            s = (s * ps) / float(ctx.q[lv - 1])
        assert len(levels) == len(pts)
        return y, s
    re = ctx.add(x, xc)
    im = ctx.mul_plain(ctx.add(xc, ctx.mul_int(x, -1)), monomial(ctx, lv))
    parts = []
    for v in (re, im):
        c = OF.cheb_encrypted(ctx, v, s, plan.coeffs, rlk)
        sc = s
        for _ in range(plan.r):
            c, sc = double_angle(ctx, c, sc, rlk)
        parts.append(c)
    s = sc
    if trace is not None:
        trace["evalmod"] = parts
    y = ctx.add(parts[0], ctx.mul_plain(parts[1], monomial(ctx, parts[1].shape[1])))
    for i, (rr, groups, ps, lv) in enumerate(plan.stc):
        y = OF.linear_encrypted(ctx, y, rr, groups, pts[len(plan.cts) + i], keys)
        s = (s * ps) / float(ctx.q[lv - 1])
    assert len(levels) == len(pts)
    return y, s
