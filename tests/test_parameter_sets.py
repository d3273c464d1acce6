"""The bootstrapping parameter sets against the reasoning behind them: the
bootstrap (default range K, doublings, degree-27 series, 3 + 3 transform
levels) leaves the stated level; SlotToCoeff's primes are at most 50 bits
(its first level's vectors carry q_0 / (2 pi Delta) ~ 2^9.4, which must stay
below 2^63 once encoded at q_{l-1}); EvalMod's and CoeffToSlot's are 60 bits;
P is at least as large as every digit; q_0 is 2^12 above the scale."""
import math

import pytest

from oracle import boot as B
from paper_2510_03996_gb300 import synth


@pytest.mark.parametrize("name,out_level", [("boot_n12", 3), ("resnet_n12", 11), ("resnet_n16", 17)])
def test_bootstrap_leaves_the_stated_level(name, out_level):
    P = synth.params(name)
    N = 1 << P["logN"]
    q = P["qbits"]
    L = len(q)
    K = B.default_K(N)
    r = B.default_doublings(K)
    depth = B.depth(3, 3, B.BOOT_DEGREE, r)
    assert L - depth == out_level
    # SlotToCoeff uses the primes just above the output level, then EvalMod, then CoeffToSlot
    stc = q[out_level:out_level + 3]
    rest = q[out_level + 3:]
    assert max(stc) <= 50 and all(b == 60 for b in rest)
    assert q[0] - math.log2(P["scale"]) == 12
    # the layers' primes below are the scale's size
    assert all(b == 40 for b in q[1:out_level])
    # SlotToCoeff's first vectors: |v| <= q_0 / (2 pi Delta), encoded at q_{l-1}
    assert math.log2(2.0 ** q[0] / (2 * math.pi * P["scale"])) + max(stc) < 62


@pytest.mark.parametrize("name", ["boot_n12", "resnet_n12", "resnet_n16", "lenet_n15", "relu_n12", "rot_n16"])
def test_special_primes_cover_every_digit(name):
    P = synth.params(name)
    q = P["qbits"]
    alpha = math.ceil(len(q) / P["dnum"])
    digits = [sum(q[j:j + alpha]) for j in range(0, len(q), alpha)]
    # bit sizes: P and each digit are products of primes just below 2^bits
    assert sum(P["pbits"]) >= max(digits)
