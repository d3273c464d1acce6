"""Host side of the LeNet-5 runner: its FP64 forward pass (used to choose the
ReLU bounds) against the oracle's plain FP64 layers, and the level budget."""
import numpy as np

from oracle import fheon as OF
from paper_2510_03996_gb300 import lenet, synth


def test_fp64_forward_matches_the_oracle_layers():
    w = lenet.weights(synth.SEED_BASE + 2)
    for s in range(3):
        X = synth.image(90, s, (1, 28, 28))
        assert np.max(np.abs(lenet.forward_fp64(X, w) - OF.lenet_fp64(X, w))) < 1e-12


def test_level_budget_and_bounds():
    P = synth.params("lenet_n15")
    assert lenet.levels() == 7 + 4 * (OF.cheb_depth(59) + 1) and len(P["qbits"]) >= lenet.levels() + 2
    w = lenet.weights(synth.SEED_BASE + 2)
    xs = [synth.image(91, s, (1, 28, 28)) for s in range(4)]
    betas = lenet.relu_bounds(xs, w)
    assert len(betas) == 4 and all(b >= 1.0 for b in betas)
    # every ReLU input of the calibration set lies inside [-beta/1.5, beta/1.5]
    for X in xs:
        rec = []
        lenet.forward_fp64(X, w, record=rec)
        assert all(np.max(np.abs(r)) * 1.5 <= b + 1e-12 for r, b in zip(rec, betas))
