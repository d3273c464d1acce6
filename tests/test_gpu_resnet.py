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


def test_mini_resnet_bit_exact_against_the_oracle():
    """The reduced network end to end, every layer from the oracle's plans and
    integer plaintexts on both sides (the library through its plain-plaintext
    layers, the oracle through its own operations), bootstraps placed by the
    same rule: the same output ciphertext to the bit."""
    from oracle import boot as B
    pr = gpu_common.Pair("resnet_n12")
    g, o = pr.g, pr.o
    N, n, D = pr.N, pr.N // 2, pr.P["scale"]
    q = [int(x) for x in g.moduli]
    w = R.weights(0xD30, MINI)
    betas = R.relu_bounds([synth.image(0xD31, i, (3, 8, 8), dist="normal") for i in range(3)], w, MINI)
    plans = {"full": B.Plan(o, D), "masked": B.Plan(o, D, slots=N // 4),
             "unmasked": B.Plan(o, D, slots=N // 4, masked=False)}
    Bl = plans["full"].out_level
    assert all(p_.out_level == Bl for p_ in plans.values())
    depth = OF.cheb_depth(R.RELU_DEGREE)
    steps = set()
    for p_ in plans.values():
        steps |= set(p_.steps())
    ops = []

    def shared(v, lv, scale):
        m = ckks.encode(v, N, scale)
        return g.plain_from_coeffs(m, lv, scale), o.plain_from_coeffs(m, lv)

    def linear(r, groups, lv, bias=None, fold=()):
        gp, op = [], []
        for _, vals in groups:
            row = [None if v is None else shared(v, lv, float(q[lv - 1])) for v in vals]
            gp.append([x and x[0] for x in row])
            op.append([x and x[1] for x in row])
        gb, ob = shared(bias, lv - 1, D) if bias is not None else (None, None)
        layer = g.linear_prepare_plain(r, [G for G, _ in groups], gp, lv, bias=gb, fold=fold)
        layer.keep = (gp, gb)
        steps.update(OF.linear_steps(r, groups))
        steps.update(f for f in fold if f)
        ops.append(("linear", layer, (r, groups, op, ob, list(fold))))

    def conv(name, m, lv, beta, stride=1, pad=1):
        K, b = w[name]
        C, H, W_, grid, dil, block = m
        F_, _, k, _ = K.shape
        r, groups = OF.conv_plan(C, F_, k, pad, H, W_, grid, dil, block, n, K / beta, stride=stride)
        Ho, Wo = (H + 2 * pad - k) // stride + 1, (W_ + 2 * pad - k) // stride + 1
        om = (F_, Ho, Wo, grid, dil * stride, block)
        bias = np.zeros(n)
        for f in range(F_):
            bias[OF.map_slots(1, Ho, Wo, grid, dil * stride, block) + f * block] = b[f] / beta
        linear(r, groups, lv, bias)
        return om

    def relu(i, lv, after, m, clean):
        # a map within slots [0, N/4) takes the sparse bootstrap: unmasked on
        # a convolution's output (zero outside its map), masked at level >= 2
        if lv - depth - after < 1:
            C_, _, _, _, _, block_ = m
            fits = C_ * block_ <= N // 4
            ops.append(("boot", "unmasked" if fits and clean else ("masked" if fits and lv >= 2 else "full")))
            lv = Bl
        ops.append(("series", OF.relu_cheb_coeffs(betas[i], R.RELU_DEGREE), lv))
        return lv - depth

    mp = R.maps(MINI)

    def compact(src, lv):
        # stage 2's strided map into its compact layout: two repack levels
        for a, b in ((src, mp["s1_rows"]), (mp["s1_rows"], mp["s1_packed"])):
            rr, gg = OF.repack_plan(*a[:3], a[3:], b[3:], n)
            linear(rr, gg, lv)
            lv -= 1
        return lv

    lv, r_i = Bl, 0
    m = conv("conv0", mp["input"], lv, betas[0])
    ops.append(("mov", "h", "x"))
    lv = relu(0, lv - 1, 1, m, True)
    r_i = 1
    bl = R.blocks(MINI)
    for bi, (s, b, ci, co, st) in enumerate(bl):
        name = "s%db%d" % (s, b)
        nxt = bl[bi + 1] if bi + 1 < len(bl) else None
        after_last = 2 if nxt is None else (3 if (nxt[0] == 1 and nxt[1] == 0) else 1)
        packs = s == 1 and b == 0   # stage 2's first block compacts both paths
        x_level, x_map = lv, m
        ops.append(("save_x",))
        ma = conv(name + "_a", m, lv, betas[r_i], stride=st)
        lv -= 1
        if packs:
            lv = compact(ma, lv)
            ma = mp["s1_packed"]
        lv = relu(r_i, lv, 1, ma, True)
        r_i += 1
        mb = conv(name + "_b", ma, lv, betas[r_i])
        lv -= 1
        sl = x_level - 1
        if st == 2:
            ops.append(("shortcut_conv",))
            msc = conv(name + "_sc", x_map, x_level, betas[r_i], stride=2, pad=0)
            if packs:
                sl = compact(msc, sl)
        else:
            ops.append(("shortcut_scale", 1.0 / betas[r_i]))
        lv = min(lv, sl)
        ops.append(("add", lv))
        lv = relu(r_i, lv, after_last, mb, st == 2)
        r_i += 1
        m = mb
    C, H, W_, grid, dil, block = m
    rr, gg = OF.avgpool_plan(C, H, H, H, W_, grid, dil, block, n)
    linear(rr, gg, lv)
    lv -= 1
    pm = (C, 1, 1, grid, dil * H, block)
    Wf, bf = w["fc"]
    fold, rr, gg = OF.fc_diag_plan(Wf, *pm, n)
    fb = np.zeros(n)
    fb[:len(bf)] = bf
    linear(rr, gg, lv, fb, fold)
    # keys and the bootstrap (composed from the oracle plan's integers)
    pr.add_keys(sorted(steps))
    conj = 2 * N - 1
    g.galois_keygen(pr.sk, [conj])
    oconj = o.rotkey(pr.s_eval, conj)
    g.relinkeygen(pr.sk)
    orlk = o.relinkey(pr.s_eval)
    okeys = {st: pr.okeys[g.galois_elt(st)] for st in steps}
    boots = {}
    for kind, pl in plans.items():
        sparse = pl.ns < pl.n
        bl_layers, bpts = [], []
        for rr_, groups, ps, blv in pl.cts + pl.stc:
            gp, op = [], []
            for _, vals in groups:
                row = [None if v is None else shared(v, blv, ps) for v in vals]
                gp.append([x and x[0] for x in row])
                op.append([x and x[1] for x in row])
            layer = g.linear_prepare_plain(rr_, [G for G, _ in groups], gp, blv)
            layer.keep = gp
            bl_layers.append(layer)
            bpts.append(op)
        prm = pr.F.fheon_boot_params(len(pl.cts), len(pl.stc), pl.K, pl.D, pl.r, 0, pl.ns if sparse else 0,
                                     0 if pl.masked else 1)
        boot = g.bootstrap_compose(prm, bl_layers[:len(pl.cts)], bl_layers[len(pl.cts):], pl.coeffs, D)
        omask = None
        if sparse and pl.masked:
            gm, omask = shared(pl.mask_slots(), 2, float(q[1]))
            g.bootstrap_set_mask(boot, gm)
        boots[kind] = (boot, pl, bpts, omask)
    used = [op[1] for op in ops if op[0] == "boot"]
    assert len(used) == 6 and "full" not in used and "unmasked" in used and "masked" in used
    # run both sides
    X = synth.image(0xD32, 0, (3, 8, 8), dist="normal")
    ct, oct_ = pr.encrypt_both(ckks.encode(R.pack_input(X, n, MINI), N, D), nonce=0xD32, level=Bl)
    G, O = {"x": ct}, {"x": oct_}
    cur = "x"
    for op in ops:
        kind = op[0]
        if kind == "linear":
            layer, (rr_, groups, opts, ob, fold) = op[1], op[2]
            G["h"] = g.layer_apply(layer, G[cur])
            y = OF.fold_encrypted(o, O[cur], fold, okeys)
            y = OF.linear_encrypted(o, y, rr_, groups, opts, okeys)
            O["h"] = o.add_plain(y, ob) if ob is not None else y
            cur = "h"
        elif kind == "series":
            _, coeffs, slv = op
            sc = g.ct_info(G[cur])[1]
            lay = g.cheb_prepare(coeffs, slv)
            G["h"] = g.layer_apply(lay, G[cur])
            O["h"] = OF.cheb_encrypted(o, O[cur], sc, coeffs, orlk)
            cur = "h"
        elif kind == "boot":
            boot, pl, bpts, omask = boots[op[1]]
            G[cur] = g.layer_apply(boot, G[cur])
            O[cur], _ = B.bootstrap_encrypted(o, O[cur], pl, bpts, okeys, orlk, oconj, mask=omask)
        elif kind == "mov":
            G[op[2]], O[op[2]] = G[op[1]], O[op[1]]
        elif kind == "save_x":
            G["x"], O["x"] = G[cur], O[cur]
            cur = "x"
        elif kind == "shortcut_scale":
            sc = g.ct_info(G["x"])[1]
            G["s"] = g.mul_const_rescale(G["x"], op[1], D)
            O["s"] = o.mul_const_rescale(O["x"], op[1], D, sc)
            G["main"], O["main"] = G[cur], O[cur]
        elif kind == "shortcut_conv":
            G["main"], O["main"] = G[cur], O[cur]
            cur = "x"   # the next linear op is the shortcut conv on the block input
        elif kind == "add":
            lv_ = op[1]
            if cur == "h" and "main" in G and G["main"] is not G["h"]:
                G["s"], O["s"] = G["h"], O["h"]      # the shortcut conv's output
            a_g, a_o = G["main"], O["main"]
            G["h"] = g.add(g.drop_level(a_g, lv_), g.drop_level(G["s"], lv_))
            O["h"] = o.add(o.drop_level(a_o, lv_), o.drop_level(O["s"], lv_))
            G.pop("main")
            cur = "h"
    assert gpu_common.mismatch(g.ct_download(G[cur]), O[cur]) == 0
    logits = np.asarray(g.decode(g.decrypt(pr.sk, G[cur]))).real[:MINI["classes"]]
    want = OF.resnet_fp64(X, w, MINI["chans"], MINI["blocks"], betas=betas)
    assert np.max(np.abs(logits - want)) < 1e-2 * max(1.0, np.max(np.abs(want)))
