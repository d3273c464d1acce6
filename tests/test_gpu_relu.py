"""The approximate ReLU (paper Sec. 5.6, Alg. 4) on the GPU against the
oracle's evaluation plan: same coefficients to the bit, same ciphertexts to the
bit from the same integer mask plaintext and input; the decrypted output
against the FP64 Chebyshev series; argument errors."""
import numpy as np
import pytest

import gpu_common
from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    pr = gpu_common.Pair("relu_n12")
    pr.g.relinkeygen(pr.sk)
    pr.orlk = pr.o.relinkey(pr.s_eval)
    return pr


@pytest.mark.parametrize("beta,D", [(4.0, 59), (2.5, 27), (1.0, 15)])
def test_coefficients_identical(beta, D):
    from paper_2510_03996_gb300 import fheon as F
    assert np.array_equal(F.relu_coeffs(beta, D), OF.relu_cheb_coeffs(beta, D))


def _input(pr, beta, n, nonce):
    x = np.zeros(pr.N // 2)
    x[:n] = synth.uniform_slots(70 + nonce, 0, n, -beta, beta)
    m = ckks.encode(x, pr.N, pr.P["scale"])
    ct, oct_ = pr.encrypt_both(m, nonce=nonce)
    return x, ct, oct_


@pytest.mark.parametrize("beta,D", [(4.0, 59), (1.0, 15)])
def test_relu_bit_exact(pair, beta, D):
    g, o = pair.g, pair.o
    n = 300
    x, ct, oct_ = _input(pair, beta, n, 1 + int(beta))
    L = pair.L
    qm = float(g.moduli[L - 1])
    mask_int = ckks.encode(OF.relu_mask_values(pair.N // 2, beta, n), pair.N, qm)
    gmask = g.plain_from_coeffs(mask_int, L, qm) if beta > 1 else None
    omask = o.plain_from_coeffs(mask_int, L) if beta > 1 else None
    layer = g.relu_prepare_plain(beta, D, gmask, L)
    y = g.relu_apply(layer, ct)
    want, _ = OF.relu_encrypted(o, oct_, pair.P["scale"], beta, D, omask, pair.orlk)
    assert gpu_common.mismatch(g.ct_download(y), want) == 0
    lv, sc = g.ct_info(y)
    assert lv == want.shape[1] and sc == pair.P["scale"]


def test_relu_decodes_to_the_series(pair):
    g = pair.g
    beta, n = 4.0, 500
    x, ct, _ = _input(pair, beta, n, 9)
    y = g.relu_approx(ct, beta, 59, n)
    got = np.asarray(g.decode(g.decrypt(pair.sk, y))).real
    want = OF.relu_fp64(x[:n], beta, 59)
    assert np.max(np.abs(got[:n] - want)) < 1e-4 * beta
    assert np.max(np.abs(got[:n] - np.maximum(0.0, x[:n]))) < 0.01 * beta


def test_relu_errors(pair):
    g, F = pair.g, pair.F
    with pytest.raises(F.FheonError) as e:
        g.relu_prepare(4.0, 59, 10, OF.cheb_depth(59) + 1)  # needs level > depth + mask
    assert e.value.code == -4
    with pytest.raises(F.FheonError) as e:
        g.relu_prepare_plain(4.0, 59, None, pair.L)  # beta > 1 needs the mask
    assert e.value.code == -1
    with pytest.raises(F.FheonError) as e:
        g.relu_prepare(-1.0, 59, 10, pair.L)
    assert e.value.code == -1
