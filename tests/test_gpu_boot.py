"""CKKS bootstrapping on the GPU against the oracle: ModRaise and the
conjugation bit for bit; the whole bootstrap bit for bit when it is composed
from the oracle's integer plaintexts; the library's own prepared bootstrap
(its own diagonals, encoded on the device) against the input message; the
one-shot call; argument and level errors."""
import numpy as np
import pytest

import gpu_common
from oracle import boot as B
from oracle import ckks
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def boot():
    pr = gpu_common.Pair("boot_n12")
    g, o = pr.g, pr.o
    plan = B.Plan(o, pr.P["scale"])
    pr.add_keys(plan.steps())
    conj = 2 * pr.N - 1
    g.galois_keygen(pr.sk, [conj])
    pr.oconj = o.rotkey(pr.s_eval, conj)
    g.relinkeygen(pr.sk)
    pr.orlk = o.relinkey(pr.s_eval)
    pr.plan = plan
    return pr


def _input(pr, seed, level):
    z = synth.uniform_slots(seed, 0, pr.N // 2)
    m = ckks.encode(z, pr.N, pr.P["scale"])
    ct, oct_ = pr.encrypt_both(m, nonce=seed, level=level)
    return z, ct, oct_


def test_mod_raise_bit_exact(boot):
    g, o = boot.g, boot.o
    for level in (1, 3):
        _, ct, oct_ = _input(boot, 0xB101 + level, level)
        r = g.mod_raise(ct)
        assert g.ct_info(r)[0] == boot.L
        want = B.mod_raise(o, o.drop_level(oct_, 1))
        assert gpu_common.mismatch(g.ct_download(r), want) == 0


def test_conjugation_bit_exact(boot):
    g, o = boot.g, boot.o
    _, ct, oct_ = _input(boot, 0xB102, 7)
    y = g.rotate_galois(ct, 2 * boot.N - 1)
    want = o.rotate(oct_, 2 * boot.N - 1, boot.oconj)
    assert gpu_common.mismatch(g.ct_download(y), want) == 0


def _composed(pr, plan=None):
    """The library's bootstrap over the oracle plan's integer plaintexts."""
    g, o = pr.g, pr.o
    plan = plan or pr.plan
    gl, opts = [], []
    for rr, groups, ps, lv in plan.cts + plan.stc:
        gp, op = [], []
        for _, vals in groups:
            grow, orow = [], []
            for v in vals:
                if v is None:
                    grow.append(None)
                    orow.append(None)
                    continue
                m = ckks.encode(v, pr.N, ps)
                grow.append(g.plain_from_coeffs(m, lv, ps))
                orow.append(o.plain_from_coeffs(m, lv))
            gp.append(grow)
            op.append(orow)
        layer = g.linear_prepare_plain(rr, [G for G, _ in groups], gp, lv)
        layer.pts = gp  # the plaintexts outlive the layer
        gl.append(layer)
        opts.append(op)
    prm = pr.F.fheon_boot_params(len(plan.cts), len(plan.stc), plan.K, plan.D, plan.r, 0,
                                 0 if plan.ns == plan.n else plan.ns, 0 if plan.masked else 1)
    return g.bootstrap_compose(prm, gl[:len(plan.cts)], gl[len(plan.cts):], plan.coeffs, pr.P["scale"]), opts


def test_bootstrap_bit_exact(boot):
    g, o, plan = boot.g, boot.o, boot.plan
    layer, opts = _composed(boot)
    okeys = {st: boot.okeys[g.galois_elt(st)] for st in plan.steps()}
    z, ct, oct_ = _input(boot, 0xB103, 2)
    y = g.layer_apply(layer, ct)
    want, osc = B.bootstrap_encrypted(o, oct_, plan, opts, okeys, boot.orlk, boot.oconj)
    assert gpu_common.mismatch(g.ct_download(y), want) == 0
    lv, sc = g.ct_info(y)
    assert lv == plan.out_level and sc == osc
    got = np.asarray(g.decode(g.decrypt(boot.sk, y))).real
    assert np.max(np.abs(got - z)) < 1e-4


def test_bootstrap_prepared_by_the_library(boot):
    g, plan = boot.g, boot.plan
    layer = g.bootstrap_prepare(boot.P["scale"])
    assert sorted(g.layer_rotation_steps(layer)) == plan.steps()
    lv, sc = g.bootstrap_info(layer)
    assert lv == plan.out_level and abs(sc / boot.P["scale"] - 1) < 1e-9
    g.bootstrap_keygen(boot.sk, layer)
    z, ct, _ = _input(boot, 0xB104, 1)
    y = g.layer_apply(layer, ct)
    assert g.ct_info(y)[0] == plan.out_level
    got = np.asarray(g.decode(g.decrypt(boot.sk, y))).real
    assert np.max(np.abs(got - z)) < 1e-4
    # the one-shot call prepares the same layer: the same ciphertext to the bit
    y1 = g.bootstrap(ct)
    assert gpu_common.mismatch(g.ct_download(y1), g.ct_download(y)) == 0
    # a bootstrapped ciphertext computes on: the output times itself, rescaled
    sq = g.rescale(g.mul_relin(y, y))
    got2 = np.asarray(g.decode(g.decrypt(boot.sk, sq))).real
    assert np.max(np.abs(got2 - z * z)) < 1e-3


def test_bootstrap_errors(boot):
    g, F = boot.g, boot.F
    layer = g.bootstrap_prepare(boot.P["scale"])
    _, ct, _ = _input(boot, 0xB105, 3)
    ct2 = g.mul_const_rescale(ct, 1.0, boot.P["scale"] * 2.0)
    with pytest.raises(F.FheonError) as e:
        g.layer_apply(layer, ct2)                 # prepared for another scale
    assert e.value.code == -5
    p = g.boot_params_default()
    assert (p.K, p.doublings, p.degree, p.cts_levels, p.stc_levels) == (plan_k(boot), boot.plan.r, 27, 3, 3)
    p.doublings = 30                                # deeper than the context
    with pytest.raises(F.FheonError) as e:
        g.bootstrap_prepare(boot.P["scale"], p)
    assert e.value.code == -4
    small = gpu_common.Pair("relu_n12")
    with pytest.raises(F.FheonError) as e:
        small.g.bootstrap_prepare(small.P["scale"])
    assert e.value.code == -4


def plan_k(pr):
    return pr.plan.K


def test_evalmod_coefficients_match_the_oracle(boot):
    for K, r, D in ((128, 7, 27), (512, 9, 27), (64, 5, 31)):
        a = boot.g.evalmod_coeffs(K, r, D)
        b = B.evalmod_coeffs(K, r, D)
        assert np.array_equal(a, b)


def test_bootstrap_batch_equals_one_by_one(boot):
    """Two inputs bootstrapped as one batch (every level, the conjugations,
    the series and the doublings batched) give each the ciphertext the
    bootstrap gives it alone, bit for bit."""
    g = boot.g
    layer = g.bootstrap_prepare(boot.P["scale"])
    g.bootstrap_keygen(boot.sk, layer)
    cts = [_input(boot, 0xB106 + i, 1 + i)[1] for i in range(2)]
    alone = [g.ct_download(g.layer_apply(layer, c)) for c in cts]
    outs = g.layer_apply_batch(layer, cts)
    for o, a in zip(outs, alone):
        assert gpu_common.mismatch(g.ct_download(o), a) == 0
    # and once more (the batch's working sets are kept and reused)
    outs = g.layer_apply_batch(layer, cts[::-1])
    for o, a in zip(outs, alone[::-1]):
        assert gpu_common.mismatch(g.ct_download(o), a) == 0


# ---------------------------------------------------------------- sparse bootstrap
@pytest.fixture(scope="module")
def sparse(boot):
    """The sparse bootstrap of slots [0, N/4) on the same context."""
    boot.splan = B.Plan(boot.o, boot.P["scale"], slots=boot.N // 4)
    boot.add_keys(boot.splan.steps())
    return boot


def test_sparse_bootstrap_bit_exact(sparse):
    """Composed from the oracle's integer plaintexts and its input mask: the
    same ciphertext to the bit as the oracle's sparse bootstrap, and the
    message of slots [0, N/4) in both copies."""
    g, o, plan = sparse.g, sparse.o, sparse.splan
    layer, opts = _composed(sparse, plan)
    mc = ckks.encode(plan.mask_slots(), sparse.N, float(o.q[1]))
    mask = g.plain_from_coeffs(mc, 2, float(o.q[1]))
    m = o.plain_from_coeffs(mc, 2)
    g.bootstrap_set_mask(layer, mask)
    assert sorted(g.layer_rotation_steps(layer)) == plan.steps()
    okeys = {st: sparse.okeys[g.galois_elt(st)] for st in plan.steps()}
    z, ct, oct_ = _input(sparse, 0xB201, 3)
    y = g.layer_apply(layer, ct)
    want, osc = B.bootstrap_encrypted(o, oct_, plan, opts, okeys, sparse.orlk, sparse.oconj, mask=m)
    assert gpu_common.mismatch(g.ct_download(y), want) == 0
    assert g.ct_info(y) == (plan.out_level, osc)
    got = np.asarray(g.decode(g.decrypt(sparse.sk, y))).real
    ns = plan.ns
    assert np.max(np.abs(got - np.tile(z[:ns], 2))) < 1e-4


def test_sparse_bootstrap_prepared_by_the_library(sparse):
    """The library's own sparse bootstrap: the oracle plan's keys, the input's
    slots [0, N/4) in both copies within 1e-4, whatever the other slots held;
    a batch equal to one by one bit for bit; an input at level 1 refused."""
    g, F, plan = sparse.g, sparse.F, sparse.splan
    p = g.boot_params_default()
    p.slots = sparse.N // 4
    layer = g.bootstrap_prepare(sparse.P["scale"], p)
    assert sorted(g.layer_rotation_steps(layer)) == plan.steps()
    assert g.bootstrap_info(layer)[0] == plan.out_level
    g.bootstrap_keygen(sparse.sk, layer)
    ns = plan.ns
    cts, zs = [], []
    for i in range(2):
        z, ct, _ = _input(sparse, 0xB202 + i, 2 + i)
        cts.append(ct)
        zs.append(z)
    alone = []
    for z, ct in zip(zs, cts):
        y = g.layer_apply(layer, ct)
        got = np.asarray(g.decode(g.decrypt(sparse.sk, y))).real
        assert np.max(np.abs(got - np.tile(z[:ns], 2))) < 1e-4
        alone.append(g.ct_download(y))
    outs = g.layer_apply_batch(layer, cts)
    for y, a in zip(outs, alone):
        assert gpu_common.mismatch(g.ct_download(y), a) == 0
    _, ct1, _ = _input(sparse, 0xB204, 1)
    with pytest.raises(F.FheonError) as e:
        g.layer_apply(layer, ct1)
    assert e.value.code == -4
    p.slots = 3
    with pytest.raises(F.FheonError) as e:
        g.bootstrap_prepare(sparse.P["scale"], p)
    assert e.value.code == -1


def test_sparse_unmasked_bootstrap(sparse):
    """The unmasked sparse bootstrap (inputs zero outside slots [0, N/4), no
    mask, level 1 taken): composed from the oracle's plaintexts, bit-exact
    against the oracle; prepared by the library, the input's slots back in
    both copies within 1e-4."""
    g, o, F = sparse.g, sparse.o, sparse.F
    plan = B.Plan(o, sparse.P["scale"], slots=sparse.N // 4, masked=False)
    layer, opts = _composed(sparse, plan)
    with pytest.raises(F.FheonError):               # no mask to replace
        g.bootstrap_set_mask(layer, g.plain_from_coeffs(np.zeros(sparse.N, dtype=np.int64), 2))
    ns = plan.ns
    z = synth.uniform_slots(0xB205, 0, sparse.N // 2)
    z[ns:] = 0.0
    ct, oct_ = sparse.encrypt_both(ckks.encode(z, sparse.N, sparse.P["scale"]), nonce=0xB205, level=1)
    okeys = {st: sparse.okeys[g.galois_elt(st)] for st in plan.steps()}
    y = g.layer_apply(layer, ct)
    want, osc = B.bootstrap_encrypted(o, oct_, plan, opts, okeys, sparse.orlk, sparse.oconj)
    assert gpu_common.mismatch(g.ct_download(y), want) == 0
    p = g.boot_params_default()
    p.slots, p.unmasked = ns, 1
    lib = g.bootstrap_prepare(sparse.P["scale"], p)
    got = np.asarray(g.decode(g.decrypt(sparse.sk, g.layer_apply(lib, ct)))).real
    assert np.max(np.abs(got - np.tile(z[:ns], 2))) < 1e-4
    p.slots = 0                                     # unmasked needs a sparse bootstrap
    with pytest.raises(F.FheonError) as e:
        g.bootstrap_prepare(sparse.P["scale"], p)
    assert e.value.code == -1
