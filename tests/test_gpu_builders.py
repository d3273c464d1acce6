"""The library's own plan builders against the oracle, element by element.

Each builder (fheon_conv_prepare, fheon_avgpool_prepare, fheon_fc_prepare
with and without its channel fold, fheon_repack_prepare, the ReLU's mask and
coefficients, fheon_bootstrap_prepare with every CoeffToSlot / SlotToCoeff
level, its X^(N/2) plaintexts and EvalMod coefficients) is read back through
the C ABI's introspection calls and compared with the oracle's plan for the
same map and weights (paper Sec. 5.1-5.5 layers, the bootstrapping layer):

  * the same tap steps, group shifts, fold shifts, output map and levels;
  * every plaintext the builder encoded, downloaded, taken to coefficients by
    the oracle's INTT and lifted, against the oracle's own encoding of the
    oracle plan's vector: within 1 + 2^-40 max|m| per coefficient.  Both sides
    round scale * tau^-1(z) in binary64 (the library by an FFT, the oracle by
    the O(N^2) sum), so they differ by rounding only: one unit at scales near
    2^40, more for the 60-bit scales of bootstrapping, whose coefficients
    exceed 2^53; a vector moved by one slot differs by the size of the
    coefficients themselves;
  * then the layer run from the library-built plan against the oracle running
    the same plan over the library's integer plaintexts: the same ciphertext
    to the bit.

Each comparison is also shown to catch a planted one-slot shift: the oracle
vector rolled by one slot (on the CPU) must fail it."""
import numpy as np
import pytest

import gpu_common
from oracle import boot as B
from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 2.0 ** -40


@pytest.fixture(scope="module")
def pair():
    return gpu_common.Pair("relu_n12")


def lib_coeffs(pr, pt):
    """A library plaintext as integer coefficients (oracle INTT, centred lift
    from the two lowest limbs), checked consistent in every limb."""
    g, o = pr.g, pr.o
    lv, sc = g.pt_info(pt)
    limbs = g.pt_download(pt)
    res = o.to_coeff(limbs, lv)
    q0, q1 = o.q[0], o.q[1]
    inv = pow(q0, -1, q1)
    m = []
    for a, b in zip(res[0].tolist(), res[1].tolist()):
        x = a + q0 * (((b - a) * inv) % q1)
        if x > (q0 * q1) // 2:
            x -= q0 * q1
        m.append(x)
    m = np.array(m, dtype=np.int64)
    for i in range(lv):
        assert np.array_equal(np.mod(m, o.q[i]).astype(np.uint64), res[i]), "limb %d is not the same integer" % i
    return m, lv, sc


def coeffs_match(m_lib, v, N, scale):
    m_or = ckks.encode(v, N, scale)
    tol = 1 + REL_TOL * float(np.max(np.abs(m_or)))
    return float(np.max(np.abs(m_lib.astype(np.float64) - m_or.astype(np.float64)))) <= tol, m_or


def check_plain(pr, pt, v, level, scale):
    """pt (library) against the oracle vector v encoded at `scale`; a planted
    one-slot shift of v must fail.  Returns the library's integer plaintext."""
    assert pt is not None
    m, lv, sc = lib_coeffs(pr, pt)
    assert lv == level and sc == scale, (lv, level, sc, scale)
    ok, _ = coeffs_match(m, v, pr.N, scale)
    assert ok
    bad, _ = coeffs_match(m, np.roll(v, 1), pr.N, scale)
    assert not bad, "a one-slot shift of the oracle vector went unnoticed"
    return m


def check_rotsum(pr, layer, r, groups, level, scale, fold=()):
    """Plan structure and every product plaintext; returns the library's
    plaintexts as oracle evaluation-form plaintexts [g][t]."""
    plan = pr.g.layer_plan(layer)
    assert plan["kind"] == 2 and plan["level"] == level
    assert plan["r"] == list(r)
    assert plan["s"] == [s for s, _ in groups]
    assert plan["fold"] == list(fold)
    opts = []
    for gi, (_, vals) in enumerate(groups):
        row = []
        for ti, v in enumerate(vals):
            pt = pr.g.layer_plain(layer, "product", gi, ti)
            if v is None:
                assert pt is None
                row.append(None)
                continue
            m = check_plain(pr, pt, v, level, scale)
            row.append(pr.o.plain_from_coeffs(m, level))
        opts.append(row)
    return opts


def run_and_compare(pr, layer, oct_, ct, r, groups, opts, bias_pt=None, fold=()):
    steps = sorted(set(OF.linear_steps(r, groups)) | {f for f in fold if f})
    pr.add_keys(steps)
    okeys = {s: pr.okeys[pr.g.galois_elt(s)] for s in steps}
    y = pr.g.layer_apply(layer, ct)
    x = OF.fold_encrypted(pr.o, oct_, list(fold), okeys) if fold else oct_
    want = OF.linear_encrypted(pr.o, x, r, groups, opts, okeys)
    if bias_pt is not None:
        want = pr.o.add_plain(want, bias_pt)
    assert gpu_common.mismatch(pr.g.ct_download(y), want) == 0
    return y


def enc_map(pr, X, grid, dil, block, nonce, level):
    v = OF.pack_map(X, pr.N // 2, grid, dil, block)
    ct, oct_ = pr.encrypt_both(ckks.encode(v, pr.N, pr.P["scale"]), nonce=nonce, level=level)
    return ct, oct_


@pytest.mark.parametrize("C,F,k,s,p,H,grid,dil,block,babies", [
    (3, 4, 3, 2, 1, 8, 8, 1, 64, 1), (8, 8, 3, 1, 1, 4, 4, 1, 16, 2), (4, 8, 1, 2, 0, 8, 8, 1, 64, 4),
    (8, 8, 3, 1, 1, 2, 4, 2, 16, 2)])
def test_conv_builder(pair, C, F, k, s, p, H, grid, dil, block, babies):
    """fheon_conv_prepare: 3 -> 4 channels, 3x3, stride 2, pad 1, with bias;
    8 -> 8 channels (block shifts by baby steps of 2 and giant steps); a 1x1
    stride-2 convolution 4 -> 8 (baby steps of 4); 8 -> 8 on a dilated map
    whose taps span more than a block (shared baby-step taps merged)."""
    pr = pair
    level = 6
    assert OF.conv_baby(k, C, F) == babies
    X = synth.image(90, 0, (C, H, H))
    K = synth.conv_kernel(90, 1, (F, C, k, k), std=0.3)
    b = synth.image(90, 2, (F,), dist="normal") * 0.1
    layer = pr.g.conv_prepare((C, H, H, grid, dil, block), K, p, level, pr.P["scale"], bias=b, stride=s)
    n = pr.N // 2
    r, groups = OF.conv_plan(C, F, k, p, H, H, grid, dil, block, n, K, stride=s)
    Ho = (H + 2 * p - k) // s + 1
    assert pr.g.layer_out_map(layer) == (F, Ho, Ho, grid, dil * s, block)
    opts = check_rotsum(pr, layer, r, groups, level, float(pr.o.q[level - 1]))
    bv = np.zeros(n)
    for f in range(F):
        bv[OF.map_slots(1, Ho, Ho, grid, dil * s, block) + f * block] = b[f]
    mb = check_plain(pr, pr.g.layer_plain(layer, "bias"), bv, level - 1, pr.P["scale"])
    ct, oct_ = enc_map(pr, X, grid, dil, block, 9000, level)
    run_and_compare(pr, layer, oct_, ct, r, groups, opts, bias_pt=pr.o.plain_from_coeffs(mb, level - 1))


def test_avgpool_builder(pair):
    pr = pair
    C, k, s, H = 2, 2, 2, 8
    grid, dil, block, level = 8, 1, 64, 5
    layer = pr.g.avgpool_prepare((C, H, H, grid, dil, block), k, s, level)
    r, groups = OF.avgpool_plan(C, k, s, H, H, grid, dil, block, pr.N // 2)
    Ho = (H - k) // s + 1
    assert pr.g.layer_out_map(layer) == (C, Ho, Ho, grid, dil * s, block)
    opts = check_rotsum(pr, layer, r, groups, level, float(pr.o.q[level - 1]))
    X = synth.image(91, 0, (C, H, H))
    ct, oct_ = enc_map(pr, X, grid, dil, block, 9100, level)
    run_and_compare(pr, layer, oct_, ct, r, groups, opts)


@pytest.mark.parametrize("C,H,grid,dil,block,m", [(4, 4, 8, 2, 64, 10), (2, 4, 4, 1, 16, 5)])
def test_fc_builder(pair, C, H, grid, dil, block, m):
    """fheon_fc_prepare in diagonal form, with the channel fold (dilation 2)
    and without it."""
    pr = pair
    level = 5
    Wm = synth.image(92, C, (m, C * H * H), dist="normal") * 0.2
    bias = synth.image(92, 7, (m,), dist="normal") * 0.1
    layer = pr.g.fc_prepare((C, H, H, grid, dil, block), Wm, level, pr.P["scale"], bias=bias)
    n = pr.N // 2
    fold, r, groups = OF.fc_diag_plan(Wm, C, H, H, grid, dil, block, n)
    assert bool(fold) == (dil > 1)
    assert pr.g.layer_out_map(layer) == (1, 1, m, m, 1, m)
    opts = check_rotsum(pr, layer, r, groups, level, float(pr.o.q[level - 1]), fold=fold)
    bv = np.zeros(n)
    bv[:m] = bias
    mb = check_plain(pr, pr.g.layer_plain(layer, "bias"), bv, level - 1, pr.P["scale"])
    X = synth.image(92, 0, (C, H, H))
    ct, oct_ = enc_map(pr, X, grid, dil, block, 9200 + C, level)
    run_and_compare(pr, layer, oct_, ct, r, groups, opts, bias_pt=pr.o.plain_from_coeffs(mb, level - 1), fold=fold)


def test_repack_builder(pair):
    pr = pair
    shape, src, dst, level = (4, 4, 4), (8, 2, 64), (4, 1, 16), 5
    layer = pr.g.repack_prepare(shape + src, shape + dst, level)
    r, groups = OF.repack_plan(*shape, src, dst, pr.N // 2)
    assert pr.g.layer_out_map(layer) == shape + dst
    opts = check_rotsum(pr, layer, r, groups, level, float(pr.o.q[level - 1]))
    X = synth.image(93, 0, shape, dist="normal")
    ct, oct_ = enc_map(pr, X, *src, 9300, level)
    run_and_compare(pr, layer, oct_, ct, r, groups, opts)


def test_relu_builder_mask_and_coefficients(pair):
    pr = pair
    beta, n, D, level = 2.5, 100, 59, 9
    layer = pr.g.relu_prepare(beta, D, n, level)
    assert pr.g.layer_plan(layer)["kind"] == 1
    assert np.array_equal(pr.g.layer_coeffs(layer), OF.relu_cheb_coeffs(beta, D))
    mask = OF.relu_mask_values(pr.N // 2, beta, n)
    check_plain(pr, pr.g.layer_plain(layer, "mask"), mask, level, float(pr.o.q[level - 1]))
    # beta <= 1: no mask
    assert pr.g.layer_plain(pr.g.relu_prepare(1.0, D, n, level), "mask") is None


@pytest.fixture(scope="module")
def boot():
    pr = gpu_common.Pair("boot_n12")
    pr.plan = B.Plan(pr.o, pr.P["scale"])
    return pr


def test_bootstrap_builder(boot):
    """fheon_bootstrap_prepare: every CoeffToSlot and SlotToCoeff level
    (plan and plaintexts), the X^(N/2) plaintexts, the EvalMod coefficients,
    then the bootstrap run from the library-built plaintexts against the
    oracle's bootstrap over the same integers, bit for bit."""
    pr, plan = boot, boot.plan
    g = pr.g
    layer = g.bootstrap_prepare(pr.P["scale"])
    info = g.layer_plan(layer)
    assert info["kind"] == 4 and (info["nt"], info["ng"]) == (len(plan.cts), len(plan.stc))
    assert np.array_equal(g.layer_coeffs(layer), plan.coeffs)
    assert g.bootstrap_info(layer)[0] == plan.out_level
    opts = []
    for i, (rr, groups, ps, lv) in enumerate(plan.cts + plan.stc):
        sub = g.layer_sub(layer, i)
        opts.append(check_rotsum(pr, sub, rr, groups, lv, ps))
    l0 = pr.L - len(plan.cts)
    l1 = l0 - OF.cheb_depth(plan.D) - plan.r
    for j, lv in enumerate((l0, l1)):
        pt = g.layer_plain(layer, "mono", j)
        assert g.pt_info(pt) == (lv, 1.0)
        assert gpu_common.mismatch(g.pt_download(pt), B.monomial(pr.o, lv)) == 0
    # the run: the library's layer against the oracle over the library's integers
    pr.add_keys(plan.steps())
    conj = 2 * pr.N - 1
    g.galois_keygen(pr.sk, [conj])
    g.relinkeygen(pr.sk)
    okeys = {st: pr.okeys[g.galois_elt(st)] for st in plan.steps()}
    z = synth.uniform_slots(0xB1D, 0, pr.N // 2)
    ct, oct_ = pr.encrypt_both(ckks.encode(z, pr.N, pr.P["scale"]), nonce=0xB1D, level=2)
    y = g.layer_apply(layer, ct)
    want, osc = B.bootstrap_encrypted(pr.o, oct_, plan, opts, okeys, pr.o.relinkey(pr.s_eval),
                                      pr.o.rotkey(pr.s_eval, conj))
    assert gpu_common.mismatch(g.ct_download(y), want) == 0
    assert g.ct_info(y) == (plan.out_level, osc)


def test_sparse_bootstrap_builder(boot):
    """fheon_bootstrap_prepare with slots = N/4: every CoeffToSlot and
    SlotToCoeff level (the N/4-slot transform in both copies, the copy factor
    in the last CoeffToSlot level, the join map in the first SlotToCoeff
    level) and the input mask against the oracle's sparse plan, then the run
    from the library-built plaintexts against the oracle over the same
    integers, bit for bit."""
    pr = boot
    g, o = pr.g, pr.o
    plan = B.Plan(o, pr.P["scale"], slots=pr.N // 4)
    p = g.boot_params_default()
    p.slots = pr.N // 4
    layer = g.bootstrap_prepare(pr.P["scale"], p)
    info = g.layer_plan(layer)
    assert (info["nt"], info["ng"]) == (len(plan.cts), len(plan.stc))
    assert g.bootstrap_info(layer)[0] == plan.out_level
    opts = []
    for i, (rr, groups, ps, lv) in enumerate(plan.cts + plan.stc):
        opts.append(check_rotsum(pr, g.layer_sub(layer, i), rr, groups, lv, ps))
    q1 = float(o.q[1])
    mm = check_plain(pr, g.layer_plain(layer, "boot_mask"), plan.mask_slots(), 2, q1)
    assert g.layer_plain(layer, "mono", 0) is None
    pr.add_keys(plan.steps())
    conj = 2 * pr.N - 1
    g.galois_keygen(pr.sk, [conj])
    g.relinkeygen(pr.sk)
    okeys = {st: pr.okeys[g.galois_elt(st)] for st in plan.steps()}
    z = synth.uniform_slots(0xB1E, 0, pr.N // 2)
    ct, oct_ = pr.encrypt_both(ckks.encode(z, pr.N, pr.P["scale"]), nonce=0xB1E, level=3)
    y = g.layer_apply(layer, ct)
    want, osc = B.bootstrap_encrypted(o, oct_, plan, opts, okeys, o.relinkey(pr.s_eval), o.rotkey(pr.s_eval, conj),
                                      mask=o.plain_from_coeffs(mm, 2))
    assert gpu_common.mismatch(g.ct_download(y), want) == 0
    assert g.ct_info(y) == (plan.out_level, osc)
