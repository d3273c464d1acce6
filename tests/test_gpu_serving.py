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


def test_one_server_two_contexts_memory_admission(setup):
    """One server takes the models of two contexts (each on its own stream):
    the results are the models' alone, bit for bit; a memory budget of one
    footprint per model keeps one request of each in flight, defers the rest
    (counted), and admits them as the earlier ones finish."""
    import torch
    pr, layers, cts, alone = setup
    g = pr.g
    model_a = g.model(layers)
    other = gpu_common.Pair("relu_n12")
    g2 = other.g
    stream = torch.cuda.Stream()
    g2.set_stream(stream.cuda_stream)
    K = synth.conv_kernel(96, 0, (1, 1, 3, 3), std=0.3)
    conv = g2.conv_prepare((1, 6, 6, GRID, 1, BLOCK), K, 1, other.L, other.P["scale"])
    other.add_keys(g2.layer_rotation_steps(conv))
    model_b = g2.model([conv])
    cts_b = []
    for i in range(2):
        X = synth.image(96, 10 + i, (1, 6, 6))
        v = OF.pack_map(X, other.N // 2, GRID, 1, BLOCK)
        cts_b.append(other.encrypt_both(ckks.encode(v, other.N, other.P["scale"]), nonce=9600 + i)[0])
    alone_b = [g2.ct_download(g2.model_run(model_b, c)) for c in cts_b]
    fa = g.model_footprint(model_a, g.ct_info(cts[0])[0])
    fb = g2.model_footprint(model_b, g2.ct_info(cts_b[0])[0])
    assert fa > fb > 0  # so that two requests of model a never fit the budget together
    srv = g.server(max_active=8, mem_budget=fa + fb)
    ids = [(srv.submit(model_a, cts[k]), "a", k) for k in range(3)] + \
          [(srv.submit(model_b, cts_b[k]), "b", k) for k in range(2)]
    res = {}
    for _ in range(200):
        srv.step()
        st = srv.model_stats(model_a)
        assert st["held"] <= fa + fb
        for rid, kind, k in ids:
            if (kind, k) not in res:
                r = srv.result(rid)
                if r is not None:
                    res[(kind, k)] = (g if kind == "a" else g2).ct_download(r)
        if len(res) == len(ids):
            break
    assert len(res) == 5
    for k in range(3):
        assert gpu_common.mismatch(res[("a", k)], alone[k]) == 0
    for k in range(2):
        assert gpu_common.mismatch(res[("b", k)], alone_b[k]) == 0
    sa, sb = srv.model_stats(model_a), srv.model_stats(model_b)
    assert sa["max_batch"] == 1 and sb["max_batch"] == 1   # one footprint each fits the budget
    assert sa["mem_waits"] > 0 and sa["held"] == 0
    srv.close()
    g2.sync()
    g2.set_stream(torch.cuda.current_stream().cuda_stream)


def test_server_graph_replay_bit_exact(setup):
    """With graph replay on, a request stepping alone runs each layer as a
    captured CUDA graph on its own buffers; finished requests hand their
    buffers to the model's next request, whose steps then replay those
    graphs.  Every result is the model's on its input alone, bit for bit;
    a context on the legacy default stream is refused."""
    import torch
    pr, layers, cts, alone = setup
    g = pr.g
    model = g.model(layers)
    srv = g.server(max_active=1)
    srv.submit(model, cts[0])
    with pytest.raises(pr.F.FheonError) as e:   # the context runs on the legacy default stream
        srv.set_graphs(True)
    assert e.value.code == -1
    srv.close()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g.set_stream(stream.cuda_stream)
    try:
        srv = g.server(max_active=1)
        srv.set_graphs(True)
        for rnd in range(2):                      # the second round reuses the pooled buffers
            for k in range(len(cts)):
                rid = srv.submit(model, cts[k])
                out = None
                for _ in range(50):
                    srv.step()
                    out = srv.result(rid)
                    if out is not None:
                        break
                assert out is not None
                assert gpu_common.mismatch(g.ct_download(out), alone[k]) == 0, (rnd, k)
        assert srv.graph_replays() == 2 * len(cts) * len(layers)
        srv.close()
    finally:
        g.sync()
        g.set_stream(torch.cuda.current_stream().cuda_stream)
