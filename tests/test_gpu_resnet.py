"""ResNet-20-style encrypted inference with bootstrapping on the GPU: the
repacking layer bit for bit against the oracle's plan (same integer masks),
the library's own repack against the plain layout change, and a reduced
network (8x8 inputs, 2/4/8 channels, one block per stage, six bootstraps)
against the FP64 network with the same approximate ReLUs."""
import numpy as np
import pytest

import gpu_common
from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import resnet as R
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

MINI = dict(img=8, in_ch=3, chans=(2, 4, 8), blocks=1, classes=10)
SHAPE, SRC, DST = (4, 4, 4), (8, 2, 64), (4, 1, 64)


@pytest.fixture(scope="module")
def small():
    return gpu_common.Pair("small_n12")


def test_repack_bit_exact(small):
    pr = small
    g, o = pr.g, pr.o
    n = pr.N // 2
    r, groups = OF.repack_plan(*SHAPE, SRC, DST, n)
    pr.add_keys(OF.linear_steps(r, groups))
    L = pr.L
    q = float(g.moduli[L - 1])
    gp, op = [], []
    for _, vals in groups:
        m = [None if v is None else ckks.encode(v, pr.N, q) for v in vals]
        gp.append([None if x is None else g.plain_from_coeffs(x, L, q) for x in m])
        op.append([None if x is None else o.plain_from_coeffs(x, L) for x in m])
    X = synth.image(0xD01, 0, SHAPE, dist="normal")
    ct, oct_ = pr.encrypt_both(ckks.encode(OF.pack_map(X, n, *SRC), pr.N, pr.P["scale"]), nonce=0xD01)
    layer = g.linear_prepare_plain(r, [G for G, _ in groups], gp, L)
    y = g.layer_apply(layer, ct)
    okeys = {s: pr.okeys[g.galois_elt(s)] for s in OF.linear_steps(r, groups)}
    want = OF.linear_encrypted(o, oct_, r, groups, op, okeys)
    assert gpu_common.mismatch(g.ct_download(y), want) == 0


def test_repack_layer_moves_the_map(small):
    pr = small
    g = pr.g
    n = pr.N // 2
    src, dst = (4,) + SHAPE[1:] + SRC, (4,) + SHAPE[1:] + DST
    layer = g.repack_prepare(src, dst, pr.L)
    r, groups = OF.repack_plan(*SHAPE, SRC, DST, n)
    assert sorted(g.layer_rotation_steps(layer)) == OF.linear_steps(r, groups)
    pr.add_keys(g.layer_rotation_steps(layer))
    X = synth.image(0xD02, 0, SHAPE, dist="normal")
    ct, _ = pr.encrypt_both(ckks.encode(OF.pack_map(X, n, *SRC), pr.N, pr.P["scale"]), nonce=0xD02)
    y = g.layer_apply(layer, ct)
    v = np.asarray(g.decode(g.decrypt(pr.sk, y))).real
    assert np.max(np.abs(OF.unpack_map(v, SHAPE, *DST) - X)) < 1e-6
    mask = np.ones(n, dtype=bool)
    mask[OF.map_slots(*SHAPE, *DST)] = False
    assert np.max(np.abs(v[mask])) < 1e-6
    assert g.layer_out_map(layer) == dst


def test_mini_resnet_matches_fp64():
    pr = gpu_common.Pair("resnet_n12")
    g = pr.g
    w = R.weights(0xD10, MINI)
    calib = [synth.image(0xD11, i, (3, 8, 8), dist="normal") for i in range(4)]
    betas = R.relu_bounds(calib, w, MINI)
    net = R.EncryptedResNet(g, w, betas, pr.P["scale"], MINI)
    assert net.n_boot == 6
    net.keygen(pr.sk)
    X = synth.image(0xD12, 0, (3, 8, 8), dist="normal")
    pt = g.encode(R.pack_input(X, pr.N // 2, MINI), pr.L, pr.P["scale"])
    ct = g.drop_level(g.encrypt(pr.pk, pt, nonce=0xD12), net.in_level)
    y = net.forward(ct)
    assert g.ct_info(y)[0] == net.out_level
    logits = np.asarray(g.decode(g.decrypt(pr.sk, y))).real[:MINI["classes"]]
    want = OF.resnet_fp64(X, w, MINI["chans"], MINI["blocks"], betas=betas)
    err = np.max(np.abs(logits - want))
    print("mini resnet: max |encrypted - fp64| = %.3g (logits up to %.3g)" % (err, np.max(np.abs(want))))
    assert err < 1e-2 * max(1.0, np.max(np.abs(want)))
    # the graph replay (first call captures, second replays) gives the same
    # ciphertext; capture needs a created stream
    import torch
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g.set_stream(stream.cuda_stream)
    for _ in range(2):
        yg = net.forward_graph(ct)
        assert gpu_common.mismatch(g.ct_download(yg), g.ct_download(y)) == 0
    g.sync()
    g.set_stream(torch.cuda.current_stream().cuda_stream)
    # the network as a native model program, alone and through the server
    # mixed with a second model (the first conv and ReLU as a chain)
    model = net.model()
    yn = g.model_run(model, ct)
    assert gpu_common.mismatch(g.ct_download(yn), g.ct_download(y)) == 0
    chain = g.model([net.layers["conv0"], net._series[(betas[0], net.in_level - 1)]])
    ct2 = g.drop_level(g.encrypt(pr.pk, g.encode(R.pack_input(X * 0.5, pr.N // 2, MINI), pr.L, pr.P["scale"]),
                                 nonce=0xD13), net.in_level)
    want_chain = g.ct_download(g.model_run(chain, ct2))
    srv = g.server(max_active=4)
    ids = [(srv.submit(model, ct), "net"), (srv.submit(chain, ct2), "chain"), (srv.submit(model, ct), "net")]
    res = {}
    for _ in range(500):
        srv.step()
        for i, (rid, _) in enumerate(ids):
            if i not in res:
                r = srv.result(rid)
                if r is not None:
                    res[i] = g.ct_download(r)
        if len(res) == len(ids):
            break
    assert len(res) == 3
    for i, (_, kind) in enumerate(ids):
        assert gpu_common.mismatch(res[i], want_chain if kind == "chain" else g.ct_download(y)) == 0
    assert srv.stats()["max_batch"] >= 2
    srv.close()


def test_program_and_repack_errors(small):
    """Argument checks of model programs, the repack layer and series layers."""
    pr = small
    g, F = pr.g, pr.F
    with pytest.raises(F.FheonError) as e:          # register out of range
        g.model_program([(F.STEP_SCALE, 0, 0, 3, 0, None, 0.5)], 2, pr.P["scale"])
    assert e.value.code == -1
    with pytest.raises(F.FheonError) as e:          # an add at level 0
        g.model_program([(F.STEP_ADD, 0, 1, 0, 0, None, 0.0)], 2, pr.P["scale"])
    assert e.value.code == -1
    with pytest.raises(F.FheonError) as e:          # a constant step without a model scale
        g.model_program([(F.STEP_SCALE, 0, 0, 0, 0, None, 0.5)], 1, 0.0)
    assert e.value.code == -1
    with pytest.raises(F.FheonError) as e:          # maps of different shapes
        g.repack_prepare((4, 4, 4, 8, 2, 64), (4, 4, 2, 4, 1, 64), pr.L)
    assert e.value.code == -1
    with pytest.raises(F.FheonError) as e:          # the target layout does not fit its blocks
        g.repack_prepare((4, 4, 4, 8, 2, 64), (4, 4, 4, 4, 1, 8), pr.L)
    assert e.value.code == -1
    with pytest.raises(F.FheonError) as e:          # a series as deep as the level
        g.cheb_prepare(np.ones(28), F.cheb_depth(27))
    assert e.value.code == -4
    with pytest.raises(F.FheonError) as e:          # a level above the context's
        g.cheb_prepare(np.ones(8), pr.L + 1)
    assert e.value.code == -1 and "level" in str(e.value)
    # a program of one constant step: c * x, rescaled onto the scale
    X = synth.image(0xD20, 0, SHAPE, dist="normal")
    n = pr.N // 2
    ct, _ = pr.encrypt_both(ckks.encode(OF.pack_map(X, n, *SRC), pr.N, pr.P["scale"]), nonce=0xD20)
    m = g.model_program([(F.STEP_SCALE, 0, 0, 1, 0, None, -0.5), (F.STEP_ADD, 1, 1, 0, pr.L - 1, None, 0.0)],
                        2, pr.P["scale"])
    y = g.model_run(m, ct)
    v = np.asarray(g.decode(g.decrypt(pr.sk, y))).real
    assert np.max(np.abs(OF.unpack_map(v, SHAPE, *SRC) + X)) < 1e-6   # 2 * (-0.5 x)
