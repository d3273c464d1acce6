"""Batched layer application and the continuous-batching server: a layer on
several inputs at once equals the layer on each alone, bit for bit; requests
that arrive while others are in flight are admitted as slots free up, share
launches with them, and each result equals the model on its input alone."""
import numpy as np
import pytest

import gpu_common
from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

GRID, BLOCK = 8, 64


@pytest.fixture(scope="module")
def setup():
    pr = gpu_common.Pair("relu_n12")
    g = pr.g
    g.relinkeygen(pr.sk)
    D = pr.P["scale"]
    lv = pr.L
    K = synth.conv_kernel(95, 0, (2, 1, 3, 3), std=0.3)
    Wm = synth.image(95, 1, (3, 2 * 3 * 3), dist="normal") * 0.3
    m0 = (1, 6, 6, GRID, 1, BLOCK)
    conv = g.conv_prepare(m0, K, 1, lv, D, bias=[0.1, -0.1])
    m1 = g.layer_out_map(conv)
    relu = g.relu_prepare(2.0, 7, m1[0] * m1[5], lv - 1)         # depth 3 + 1 + 1
    pool = g.avgpool_prepare(m1, 2, 2, lv - 6)
    fc = g.fc_prepare(g.layer_out_map(pool), Wm, lv - 7, D)  # one level: ends at lv - 8
    layers = [conv, relu, pool, fc]
    for layer in layers:
        pr.add_keys(g.layer_rotation_steps(layer))
    xs = [synth.image(95, 10 + i, (1, 6, 6)) for i in range(5)]
    cts = []
    for i, X in enumerate(xs):
        v = OF.pack_map(X, pr.N // 2, GRID, 1, BLOCK)
        cts.append(pr.encrypt_both(ckks.encode(v, pr.N, D), nonce=9500 + i)[0])
    alone = []
    for ct in cts:
        y = ct
        for layer in layers:
            y = g.layer_apply(layer, y)
        alone.append(g.ct_download(y))
    return pr, layers, cts, alone


def test_batch_apply_equals_single(setup):
    pr, layers, cts, alone = setup
    g = pr.g
    ys = list(cts[:3])
    for layer in layers:
        single = [g.ct_download(g.layer_apply(layer, y)) for y in ys]
        ys = g.layer_apply_batch(layer, ys)
        for a, b in zip(ys, single):
            assert gpu_common.mismatch(g.ct_download(a), b) == 0
    with pytest.raises(pr.F.FheonError) as e:
        g.layer_apply_batch(layers[0], [cts[0], cts[1]], [cts[1], g.ct_create(1)])
    assert e.value.code == -1


def test_server_mixes_requests_bit_exactly(setup):
    pr, layers, cts, alone = setup
    g = pr.g
    model = g.model(layers)
    srv = g.server(max_active=3)
    ids = {}
    ids[0] = srv.submit(model, cts[0])
    srv.step()                                   # request 0 alone at layer 0
    ids[1] = srv.submit(model, cts[1])
    ids[2] = srv.submit(model, cts[2])
    assert srv.result(ids[1]) is None            # pending
    srv.step()
    ids[3] = srv.submit(model, cts[3])           # waits: three in flight
    ids[4] = srv.submit(model, cts[4])
    st = srv.stats()
    assert st["active"] == 3 and st["waiting"] == 2
    results = {}
    for _ in range(100):
        srv.step()
        for k, rid in ids.items():
            if k not in results:
                out = srv.result(rid)
                if out is not None:
                    results[k] = g.ct_download(out)
        if len(results) == len(ids):
            break
    assert len(results) == 5
    for k in range(5):
        assert gpu_common.mismatch(results[k], alone[k]) == 0
    assert srv.stats()["max_batch"] >= 2
    with pytest.raises(pr.F.FheonError):
        srv.result(ids[0])                        # taken already
    srv.close()
