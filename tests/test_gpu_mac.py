"""fheon_mac_plain (sum of plaintext products in one pass) against the oracle's
sequence of plaintext products and additions: bit-exact, including more terms
than one launch takes (the chunked path), and its argument errors."""
import numpy as np
import pytest

import gpu_common
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    return gpu_common.Pair("small_n12")


def _operands(pr, n, level, seed):
    cts, octs, pts, opts = [], [], [], []
    for t in range(n):
        c, oc = pr.encrypt_both(synth.small_int_poly(seed, t, pr.N, 1 << 40), nonce=4000 + seed * 100 + t, level=level)
        cts.append(c)
        octs.append(oc)
        w = synth.small_int_poly(seed + 1, t, pr.N, 1 << 20)
        pts.append(pr.g.plain_from_coeffs(w, pr.L, 2.0 ** 20))
        opts.append(pr.o.plain_from_coeffs(w, pr.L))
    return cts, octs, pts, opts


@pytest.mark.parametrize("n,level", [(1, 5), (25, 3), (40, 2)])
def test_mac_plain_bit_exact(pair, n, level):
    cts, octs, pts, opts = _operands(pair, n, level, 7 + n)
    out = pair.g.mac_plain(cts, pts)
    want = None
    for oc, op in zip(octs, opts):
        prod = pair.o.mul_plain(oc, op)
        want = prod if want is None else pair.o.add(want, prod)
    assert gpu_common.mismatch(pair.g.ct_download(out), want) == 0
    assert pair.g.ct_info(out)[0] == level


def test_mac_plain_errors(pair):
    g, F = pair.g, pair.F
    cts, _, pts, _ = _operands(pair, 2, 3, 90)
    with pytest.raises(F.FheonError) as e:
        g.mac_plain(cts, pts, out=cts[1])
    assert e.value.code == -1
    other = g.drop_level(cts[1], 2)
    with pytest.raises(F.FheonError) as e:
        g.mac_plain([cts[0], other], pts)
    assert e.value.code == -4
    w = synth.small_int_poly(91, 0, pair.N, 1 << 20)
    with pytest.raises(F.FheonError) as e:
        g.mac_plain(cts, [pts[0], g.plain_from_coeffs(w, pair.L, 2.0 ** 21)])
    assert e.value.code == -5
