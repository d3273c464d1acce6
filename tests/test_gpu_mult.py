"""Ciphertext product with relinearisation and the scalar operations on the
GPU against the oracle: the relinearisation key and every result bit-exact,
at every level of a 5-limb chain; argument errors."""
import numpy as np
import pytest

import gpu_common
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    pr = gpu_common.Pair("small_n12")
    pr.g.relinkeygen(pr.sk)
    pr.orlk = pr.o.relinkey(pr.s_eval)
    return pr


def test_relin_key(pair):
    assert gpu_common.mismatch(pair.g.key_download(0), pair.orlk) == 0


@pytest.mark.parametrize("level", [5, 4, 3, 2, 1])
def test_mul_relin_bit_exact(pair, level):
    g = pair.g
    a, oa = pair.encrypt_both(synth.small_int_poly(51, level, pair.N, 1 << 40), nonce=5000 + level, level=level)
    b, ob = pair.encrypt_both(synth.small_int_poly(52, level, pair.N, 1 << 40), nonce=5100 + level, level=level)
    want = pair.o.mul_relin(oa, ob, pair.orlk)
    out = g.mul_relin(a, b)
    assert gpu_common.mismatch(g.ct_download(out), want) == 0
    sa = g.ct_info(a)[1]
    assert g.ct_info(out) == (level, sa * g.ct_info(b)[1])
    # in place, and the square
    g.mul_relin(a, b, out=a)
    assert gpu_common.mismatch(g.ct_download(a), want) == 0
    sq = g.mul_relin(b, b)
    assert gpu_common.mismatch(g.ct_download(sq), pair.o.mul_relin(ob, ob, pair.orlk)) == 0


def test_scalar_ops_bit_exact(pair):
    g, o = pair.g, pair.o
    D = pair.P["scale"]
    ct, oct_ = pair.encrypt_both(synth.small_int_poly(53, 0, pair.N, 1 << 40), nonce=5200, level=4)
    for v in (3, -7, 1 << 45, -(1 << 55)):
        assert gpu_common.mismatch(g.ct_download(g.mul_int(ct, v)), o.mul_int(oct_, v)) == 0
        assert gpu_common.mismatch(g.ct_download(g.add_int(ct, v)), o.add_int(oct_, v)) == 0
    for c in (0.5, -1.0, 3.25e-3):
        assert gpu_common.mismatch(g.ct_download(g.add_const(ct, c)), o.add_const(oct_, c, D)) == 0
    for c, target in ((0.37, D), (-2.5, D / 3.0), (1.0, D * 0.999)):
        out = g.mul_const_rescale(ct, c, target)
        assert gpu_common.mismatch(g.ct_download(out), o.mul_const_rescale(oct_, c, target, D)) == 0
        assert g.ct_info(out) == (3, target)


def test_product_errors(pair):
    g, F = pair.g, pair.F
    a, _ = pair.encrypt_both(synth.small_int_poly(54, 0, pair.N, 1 << 40), nonce=5300, level=4)
    b, _ = pair.encrypt_both(synth.small_int_poly(54, 1, pair.N, 1 << 40), nonce=5301, level=3)
    with pytest.raises(F.FheonError) as e:
        g.mul_relin(a, b)
    assert e.value.code == -4
    one = g.drop_level(b, 1)
    with pytest.raises(F.FheonError) as e:
        g.mul_const_rescale(one, 0.5, 1.0)
    assert e.value.code == -4
    with pytest.raises(F.FheonError) as e:
        g.add_const(a, 1e300)
    assert e.value.code == -1
    other = gpu_common.Pair("small_n12")  # no relinearisation key
    x, _ = other.encrypt_both(synth.small_int_poly(55, 0, other.N, 1 << 40), nonce=1, level=2)
    with pytest.raises(F.FheonError) as e:
        other.g.mul_relin(x, x)
    assert e.value.code == -3


def test_product_decodes(pair):
    """mul_relin then rescale decodes to the slot-wise product."""
    g = pair.g
    D = pair.P["scale"]
    z1 = synth.uniform_slots(56, 0, pair.N // 2)
    z2 = synth.uniform_slots(56, 1, pair.N // 2)
    a = g.drop_level(g.encrypt(pair.pk, g.encode(z1, pair.L, D), nonce=5400), 4)
    b = g.drop_level(g.encrypt(pair.pk, g.encode(z2, pair.L, D), nonce=5401), 4)
    r = g.rescale(g.mul_relin(a, b))
    lv, sc = g.ct_info(r)
    got = g.decode(g.decrypt(pair.sk, r))
    assert lv == 3 and sc == pytest.approx(D * D / pair.g.moduli[3])
    tol = (pair.N + 1) / 2 * np.sqrt(pair.N) / sc
    assert np.max(np.abs(np.asarray(got)[: pair.N // 2].real - z1 * z2)) < tol
