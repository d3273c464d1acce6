"""Pins of the oracle's approximate ReLU (paper Sec. 5.6, Alg. 4): the
Chebyshev coefficients against numpy's Chebyshev interpolation (the same nodes,
a library routine) and the interpolation property at the nodes; the series'
distance to max(0, x); and the encrypted evaluation plan against the FP64
series under decryption."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth


@pytest.mark.parametrize("beta,D", [(1.0, 59), (4.0, 59), (2.5, 27)])
def test_coeffs_are_chebyshev_interpolation(beta, D):
    c = OF.relu_cheb_coeffs(beta, D)
    f = lambda z: np.where(z < 0, 0.0, beta * z)  # noqa: E731
    want = npcheb.chebinterpolate(f, D)
    assert np.max(np.abs(c - want)) < 1e-12 * max(1.0, beta)
    nodes = np.cos(np.pi * (np.arange(D + 1) + 0.5) / (D + 1))
    assert np.max(np.abs(OF.cheb_eval_fp64(c, nodes) - f(nodes))) < 1e-12 * max(1.0, beta)


def test_series_is_close_to_relu():
    """Degree 59 on [-beta, beta]: within 1 % of beta of max(0, x) (the kink
    at 0 limits a polynomial to O(beta / D))."""
    for beta in (1.0, 4.0):
        x = np.linspace(-beta, beta, 4001)
        err = np.abs(OF.relu_fp64(x, beta) - np.maximum(0.0, x))
        assert err.max() < 0.01 * beta
        assert err[np.abs(x) > 0.25 * beta].max() < 0.002 * beta


@pytest.fixture(scope="module")
def ctx10():
    # the ReLU test moduli at N = 2^10 to keep the oracle fast
    P = synth.params("relu_n12")
    N = 1 << 10
    mods = ckks.gen_primes(N, P["qbits"] + P["pbits"])
    L = len(P["qbits"])
    ctx = ckks.Ctx(N, mods[:L], mods[L:], P["dnum"], P["seed"])
    s, se = ctx.keygen_sk()
    return ctx, P, se, ctx.keygen_pk(se), ctx.relinkey(se)


@pytest.mark.parametrize("beta", [4.0, 1.0])
def test_encrypted_relu_matches_the_series(ctx10, beta):
    ctx, P, se, pk, rlk = ctx10
    N, D, scale = ctx.N, OF.RELU_DEGREE, P["scale"]
    n = 300
    x = np.zeros(N // 2)
    x[:n] = synth.uniform_slots(61, 0, n, -beta, beta)
    ct = ctx.encrypt(pk, ckks.encode(x, N, scale), 3)
    lvl = ct.shape[1]
    mask = ctx.plain_from_coeffs(ckks.encode(OF.relu_mask_values(N // 2, beta, n), N, float(ctx.q[lvl - 1])), lvl)
    y, sy = OF.relu_encrypted(ctx, ct, scale, beta, D, mask, rlk)
    depth = OF.cheb_depth(D) + (1 if beta > 1 else 0)
    assert y.shape[1] == lvl - depth and sy == scale
    got = ctx.decode_ct(se, y, sy).real
    want = OF.relu_fp64(x[:n], beta, D)
    assert np.max(np.abs(got[:n] - want)) < 1e-4 * beta
    if beta > 1:  # the mask zeroed the other slots: f(0) = c-series at 0
        assert np.max(np.abs(got[n:] - OF.relu_fp64(0.0, beta, D))) < 1e-4 * beta


def test_series_tree_and_depth():
    """The baby-step/giant-step tree equals the plain Chebyshev sum (the
    division p = r + q T_g), and the library's series depth is the oracle's."""
    from paper_2510_03996_gb300 import fheon as F
    z = np.linspace(-1, 1, 257)
    for D in (1, 2, 3, 7, 15, 27, 31, 59, 63, 100, 255):
        c = synth.rng(0x5E, D).normal(size=D + 1)
        assert np.max(np.abs(OF.ps_eval_fp64(c, z) - OF.cheb_eval_fp64(c, z))) < 1e-12 * D
    for D in range(1, 300):
        assert F.cheb_depth(D) == OF.cheb_depth(D), D
        assert OF.cheb_depth(D) <= int(np.ceil(np.log2(D + 1))) + 1
    assert OF.cheb_depth(59) == 6 and OF.cheb_depth(27) == 5
