"""GPU parity: every step of the rotation path through the C ABI against the
CPU oracle, residue for residue (integer work: bit-exact), on seeded inputs at
sizes that span several NTT tiles, partial last digits and level edges."""
import numpy as np
import pytest

from oracle import ckks as O
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

import gpu_common


@pytest.fixture(scope="module")
def small():
    # N = 2^12, Q = 5 limbs, P = 2 limbs, dnum = 3 -> alpha = 2, beta = 3
    return gpu_common.Pair("small_n12", rot_steps=[1, -1, 5, 100, 2047])


@pytest.fixture(scope="module")
def conv13():
    # configuration of the single-conv workload: N = 2^13, Q {60,40,40}, P {60}, dnum 3
    return gpu_common.Pair("conv_n13", rot_steps=OF.conv_rotation_steps(28, 5))


def test_moduli_match(small, conv13):
    for pr in (small, conv13):
        assert pr.g.moduli == pr.o_primes
        assert (pr.g.alpha, pr.g.beta) == (pr.o.alpha, pr.o.beta)


def test_secret_and_public_keys(small):
    assert gpu_common.mismatch(small.g.sk_download(small.sk), small.s_eval) == 0
    assert gpu_common.mismatch(small.g.pk_download(small.pk), small.opk) == 0


def test_rotation_keys(small, conv13):
    for pr in (small, conv13):
        for g, ok in pr.okeys.items():
            assert gpu_common.mismatch(pr.g.key_download(g), ok) == 0, g


def test_plaintext_from_coefficients(small):
    m = synth.small_int_poly(1, 2, small.N, 1 << 40)
    for level in (small.L, 3, 1):
        pt = small.g.plain_from_coeffs(m, level, 1.0)
        assert gpu_common.mismatch(small.g.pt_download(pt), small.o.plain_from_coeffs(m, level)) == 0


def test_encrypt_decrypt(small):
    m = synth.small_int_poly(2, 0, small.N, 1 << 35)
    ct, oct_ = small.encrypt_both(m, nonce=77)
    assert gpu_common.mismatch(small.g.ct_download(ct), oct_) == 0
    for level in (small.L, 2):
        c = small.g.drop_level(ct, level)
        dec = small.g.pt_download(small.g.decrypt(small.sk, c))
        assert gpu_common.mismatch(dec, small.o.decrypt(small.s_eval, oct_[:, :level])) == 0


@pytest.mark.parametrize("level", [5, 4, 3, 2, 1])
@pytest.mark.parametrize("step", [1, -1, 5, 100, 2047])
def test_rotate_bit_exact(small, level, step):
    m = synth.small_int_poly(3, level * 31 + (step & 0xFFF), small.N, 1 << 40)
    ct, oct_ = small.encrypt_both(m, nonce=1000 + level, level=level)
    out = small.g.rotate(ct, step)
    g = small.g.galois_elt(step)
    want = small.o.rotate(oct_, g, small.okeys[g])
    assert gpu_common.mismatch(small.g.ct_download(out), want) == 0


def test_rotate_in_place_and_batch(small):
    m = synth.small_int_poly(4, 0, small.N, 1 << 40)
    ct, oct_ = small.encrypt_both(m, nonce=5, level=5)
    g = small.g.galois_elt(5)
    want = small.o.rotate(oct_, g, small.okeys[g])
    c2 = small.g.drop_level(ct, 5)
    small.g.rotate(c2, 5, out=c2)
    assert gpu_common.mismatch(small.g.ct_download(c2), want) == 0
    # batch of mixed levels and steps equals single rotations
    ins, outs, steps, wants = [], [], [], []
    for i, (lv, st) in enumerate([(5, 1), (3, -1), (1, 100), (4, 5), (2, 2047), (5, 1)]):
        mi = synth.small_int_poly(4, 10 + i, small.N, 1 << 40)
        c, oc = small.encrypt_both(mi, nonce=200 + i, level=lv)
        ins.append(c)
        outs.append(small.g.ct_create(1))
        steps.append(st)
        gg = small.g.galois_elt(st)
        wants.append(small.o.rotate(oc, gg, small.okeys[gg]))
    small.g.rotate_batch(ins, outs, steps)
    for o, w in zip(outs, wants):
        assert gpu_common.mismatch(small.g.ct_download(o), w) == 0


def test_schedule_range(small):
    g = small.g
    old = g.get_schedule()
    try:
        for bad in (-1, 8, 10, 16):
            with pytest.raises(small.F.FheonError) as e:
                g.set_schedule(bad)
            assert e.value.code == -1
        assert g.get_schedule() == old
    finally:
        g.set_schedule(old)


@pytest.mark.parametrize("schedule", [0, 1, 2, 3, 4, 5, 6, 7, 9, 11, 13, 15, 17, 25, 31])
def test_every_schedule_is_bit_exact(small, schedule):
    """Key-switching schedules change launches and fusion only, never results:
    single rotations (closed-form tasks) and batches at mixed levels."""
    g = small.g
    old = g.get_schedule()
    g.set_schedule(schedule)
    try:
        ins, outs, steps, wants = [], [], [], []
        for i, (lv, st) in enumerate([(5, 1), (3, 5), (4, -1), (1, 2047), (2, 100)]):
            m = synth.small_int_poly(50 + schedule, i, small.N, 1 << 40)
            c, oc = small.encrypt_both(m, nonce=700 + 10 * schedule + i, level=lv)
            gg = g.galois_elt(st)
            w = small.o.rotate(oc, gg, small.okeys[gg])
            assert gpu_common.mismatch(g.ct_download(g.rotate(c, st)), w) == 0
            ins.append(c)
            outs.append(g.ct_create(1))
            steps.append(st)
            wants.append(w)
        g.rotate_batch(ins, outs, steps)
        for o, w in zip(outs, wants):
            assert gpu_common.mismatch(g.ct_download(o), w) == 0
    finally:
        g.set_schedule(old)


def test_missing_key_is_an_error(small):
    m = synth.small_int_poly(5, 0, small.N, 100)
    ct, _ = small.encrypt_both(m, nonce=9)
    with pytest.raises(small.F.FheonError) as e:
        small.g.rotate(ct, 7)
    assert e.value.code == -3


def test_mul_plain_add_rescale(small):
    g = small.g
    m1 = synth.small_int_poly(6, 0, small.N, 1 << 40)
    m2 = synth.small_int_poly(6, 1, small.N, 1 << 40)
    w = synth.small_int_poly(6, 2, small.N, 1 << 20)
    for level in (5, 3, 2):
        c1, o1 = small.encrypt_both(m1, nonce=300 + level, level=level)
        c2, o2 = small.encrypt_both(m2, nonce=400 + level, level=level)
        pt = g.plain_from_coeffs(w, level, 1.0)
        opt = small.o.plain_from_coeffs(w, level)
        assert gpu_common.mismatch(g.ct_download(g.mul_plain(c1, pt)), small.o.mul_plain(o1, opt)) == 0
        assert gpu_common.mismatch(g.ct_download(g.add(c1, c2)), small.o.add(o1, o2)) == 0
        pts = g.plain_from_coeffs(w, level, small.P["scale"])  # same scale as the ciphertext
        assert gpu_common.mismatch(g.ct_download(g.add_plain(c1, pts)), small.o.add_plain(o1, opt)) == 0
        r = g.rescale(c1)
        assert g.ct_info(r)[0] == level - 1
        assert gpu_common.mismatch(g.ct_download(r), small.o.rescale(o1)) == 0
        # in place
        c3 = g.drop_level(c1, level)
        g.rescale(c3, out=c3)
        assert gpu_common.mismatch(g.ct_download(c3), small.o.rescale(o1)) == 0


def test_level_and_scale_errors(small):
    m = synth.small_int_poly(7, 0, small.N, 100)
    a, _ = small.encrypt_both(m, nonce=1, level=3)
    b, _ = small.encrypt_both(m, nonce=2, level=2)
    with pytest.raises(small.F.FheonError) as e:
        small.g.add(a, b)
    assert e.value.code == -4
    c = small.g.rescale(small.g.drop_level(a, 3))
    with pytest.raises(small.F.FheonError) as e:
        small.g.add(c, small.g.drop_level(a, 2))
    assert e.value.code == -5


def test_encode_against_oracle(small):
    N = small.N
    z = synth.uniform_slots(8, 0, N // 2, complex_=True)
    got = small.g.encode_coeffs(z, 2.0 ** 40)
    want = O.encode(z, N, 2.0 ** 40)
    # FP64 FFT vs the O(N^2) definition: rounding may differ by one unit
    assert np.max(np.abs(got - want)) <= 1
    assert np.mean(got == want) > 0.99
    # partial slots
    got = small.g.encode_coeffs(z[:100], 2.0 ** 30)
    assert np.max(np.abs(got - O.encode(z[:100], N, 2.0 ** 30))) <= 1


def test_decode_and_rotation_semantics(small):
    g = small.g
    N = small.N
    z = synth.uniform_slots(9, 0, N // 2, complex_=True)
    pt = g.encode(z, small.L, 2.0 ** 40)
    back = g.decode(pt)
    assert np.max(np.abs(back - z)) < 1e-9
    ct = g.encrypt(small.pk, pt, nonce=3)
    for step in (1, -1, 5):
        r = g.rotate(g.drop_level(ct, 3), step)
        got = g.decode(g.decrypt(small.sk, r))
        assert np.max(np.abs(got - np.roll(z, -step))) < 1e-6


def _tap_plains_int(pr, k, level, seed):
    return [synth.small_int_poly(seed, t, pr.N, 1 << 20) for t in range(k * k)]


def test_conv2d_orchestration_bit_exact(conv13):
    """Library special conv with caller-made integer tap plaintexts vs the
    oracle's Sec. 5.3 orchestration on the same plaintexts (N = 2^13, 28x28, 5x5),
    tap rotations hoisted on both sides."""
    pr = conv13
    g = pr.g
    H = W = 28
    k = 5
    level = 3
    taps_int = _tap_plains_int(pr, k, level, 11)
    taps = [g.plain_from_coeffs(t, level, float(pr.g.moduli[level - 1])) for t in taps_int]
    otaps = [pr.o.plain_from_coeffs(t, level) for t in taps_int]
    m = synth.small_int_poly(12, 0, pr.N, 1 << 40)
    ct, oct_ = pr.encrypt_both(m, nonce=21)
    layer = g.conv2d_prepare_plain(1, k, H, W, level, taps)
    out = g.conv2d_apply(layer, ct)
    okeys = {r: pr.okeys[pr.g.galois_elt(r)] for r in OF.conv_rotation_steps(W, k)}
    want = OF.special_conv_encrypted(pr.o, oct_, okeys, H, W, k, otaps, hoisted=True)
    assert gpu_common.mismatch(g.ct_download(out), want) == 0


def test_conv2d_graph_replay_bit_exact(conv13):
    """The CUDA-graph application of a conv layer equals the eager one, on the
    first (capturing) call and on replays with new data in the same buffers."""
    import torch
    pr = conv13
    g = pr.g
    s = torch.cuda.Stream()
    g.set_stream(s.cuda_stream)
    try:
        P = pr.P
        K = synth.conv_kernel(P["seed"], 7, (1, 5, 5))
        layer = g.conv2d_prepare(1, 5, 1, 2, 28, 28, K, [0.25], pr.L, P["scale"])
        ct_in = g.ct_create(pr.L, P["scale"])
        out_graph = g.ct_create(pr.L)
        for trial in range(3):
            m = synth.small_int_poly(60 + trial, 0, pr.N, 1 << 40)
            ct, _ = pr.encrypt_both(m, nonce=900 + trial)
            host = g.ct_download(ct)
            keep = g.ct_upload(ct_in, host)
            g.sync()
            eager = g.ct_download(g.conv2d_apply(layer, ct))
            g.conv2d_apply_graph(layer, ct_in, out_graph)
            g.sync()
            assert gpu_common.mismatch(g.ct_download(out_graph), eager) == 0
            del keep
    finally:
        g.set_stream(torch.cuda.current_stream().cuda_stream)


def test_conv2d_matches_fp64(conv13):
    """Config-1 conv (1x28x28 U[0,1], 5x5 N(0, 0.1^2), pad 2) decrypts to the FP64
    convolution within 1e-5 (noise after 24 key switches and one rescale at
    scale 2^40 is ~1e-8; the tolerance leaves three orders of margin)."""
    pr = conv13
    g = pr.g
    P = pr.P
    H = W = 28
    X = synth.image(P["seed"], 0, (1, H, W))
    K = synth.conv_kernel(P["seed"], 1, (1, 1, 5, 5))
    x = np.zeros(pr.N // 2)
    x[:H * W] = X.reshape(-1)
    ct = g.encrypt(pr.pk, g.encode(x, pr.L, P["scale"]), nonce=1)
    out = g.conv2d(ct, 1, 1, 5, 1, 2, H, W, K)
    lv, sc = g.ct_info(out)
    assert lv == 2 and abs(sc - P["scale"]) / P["scale"] < 1e-12
    y = g.decode(g.decrypt(pr.sk, out)).real
    ref = OF.conv2d_fp64(X, K, pad=2).reshape(-1)
    assert np.max(np.abs(y[:H * W] - ref)) < 1e-5
    assert np.max(np.abs(y[H * W:])) < 1e-5


def test_rotate_full_size_sampled():
    """Batched-rotation workload parameters (N = 2^16, 24 x 50-bit Q, 4 x 60-bit P,
    dnum 6): whole ciphertexts at a full and a partial-digit level against the
    oracle, which is slow at this size (one key, two rotations)."""
    pr = gpu_common.Pair("rot_n16", rot_steps=[12345])
    g = pr.g.galois_elt(12345)
    assert gpu_common.mismatch(pr.g.key_download(g), pr.okeys[g]) == 0
    m = synth.small_int_poly(13, 0, pr.N, 1 << 40)
    ct, oct_ = pr.encrypt_both(m, nonce=3)
    for level in (24, 9):
        want = pr.o.rotate(oct_[:, :level], g, pr.okeys[g])
        c = pr.g.drop_level(ct, level)
        for schedule in (9, 25):  # row passes at radix 16 and at radix 8
            pr.g.set_schedule(schedule)
            out = pr.g.rotate(c, 12345)
            assert gpu_common.mismatch(pr.g.ct_download(out), want) == 0, schedule


def test_autotune_cache(small, tmp_path):
    """The autotuner's choice is saved per parameters and batch shape and reused."""
    import json
    g = small.g
    old = g.get_schedule()
    try:
        ins, outs, steps = [], [], []
        for i, (lv, st) in enumerate([(5, 1), (3, -1), (4, 5)]):
            c, _ = small.encrypt_both(synth.small_int_poly(70, i, small.N, 1 << 40), nonce=7000 + i, level=lv)
            ins.append(c)
            outs.append(g.ct_create(1))
            steps.append(st)
        path = str(tmp_path / "schedules.json")
        best, ms = g.autotune_schedule(ins, outs, steps, reps=1, cache=path)
        saved = json.load(open(path))
        assert len(saved) == 1 and list(saved.values())[0]["schedule"] == best
        g.set_schedule(0)
        best2, ms2 = g.autotune_schedule(ins, outs, steps, reps=1, cache=path)
        assert best2 == best and g.get_schedule() == best and ms2 == ms
    finally:
        g.set_schedule(old)


def test_rotate_batch_bench_configuration_sampled():
    """The benchmark's batch itself: 256 ciphertexts at N = 2^16 (24 + 4 limbs,
    dnum 6) at the workload's levels U{4..24}, each rotated by its own step
    with its own key, in one fheon_rotate_batch call under the default
    schedule; three sampled outputs (the lowest, a middle and the highest
    level) bit-exact against the oracle's rotation of the same encryption."""
    import oracle.ckks as O
    P = synth.params("rot_n16")
    levels, steps = synth.rotation_workload(P["seed"])
    pick = [int(np.argmin(levels)), len(levels) // 2, int(np.argmax(levels))]
    pr = gpu_common.Pair("rot_n16", rot_steps=[steps[i] for i in pick])
    g = pr.g
    g.galois_keygen(pr.sk, sorted({g.galois_elt(s) for s in steps}))
    m = synth.small_int_poly(P["seed"], 21, pr.N, 1 << 40)
    pt = g.plain_from_coeffs(m, pr.L, P["scale"])
    ins = [g.drop_level(g.encrypt(pr.pk, pt, nonce=i), lv) for i, lv in enumerate(levels)]
    outs = [g.ct_create(lv) for lv in levels]
    g.rotate_batch(ins, outs, steps)
    for i in pick:
        oc = pr.o.drop_level(pr.o.encrypt(pr.opk, m, i), levels[i])
        ge = O.galois_elt(steps[i], pr.N)
        want = pr.o.rotate(oc, ge, pr.okeys[ge])
        assert gpu_common.mismatch(g.ct_download(outs[i]), want) == 0, (i, levels[i], steps[i])


def test_ciphertext_batch_transfers(small):
    """A contiguous ciphertext batch: one-copy round trips through host memory,
    rotation of batch ciphertexts equal to that of ordinary ones, and the
    per-ciphertext fallback once a ciphertext's level changes."""
    g = small.g
    levels = [5, 2, 4]
    batch = g.ct_create_batch(levels, small.P["scale"])
    singles = []
    for i, (lv, b) in enumerate(zip(levels, batch)):
        c, _ = small.encrypt_both(synth.small_int_poly(71, i, small.N, 1 << 40), nonce=7100 + i, level=lv)
        g.drop_level(c, lv, out=b)
        singles.append(c)
    words = sum(2 * lv * small.N for lv in levels)
    host = np.zeros(words, dtype=np.uint64)
    g.ct_download_many_async(batch, host.ctypes.data)
    g.sync()
    off = 0
    for lv, c in zip(levels, singles):
        n = 2 * lv * small.N
        assert np.array_equal(host[off:off + n].reshape(2, lv, small.N), g.ct_download(c))
        off += n
    other = g.ct_create_batch(levels, small.P["scale"])
    g.ct_upload_many_async(other, host.ctypes.data)
    g.sync()
    outs_b = g.ct_create_batch(levels, small.P["scale"])
    g.rotate_batch(other, outs_b, [1, -1, 5])
    outs_s = [g.ct_create(1) for _ in levels]
    g.rotate_batch(singles, outs_s, [1, -1, 5])
    for a, b in zip(outs_b, outs_s):
        assert gpu_common.mismatch(g.ct_download(a), g.ct_download(b)) == 0
    # a level change breaks contiguity: the copies go one by one and stay right
    g.drop_level(other[0], 3, out=other[0])
    back = np.zeros(sum(2 * g.ct_info(c)[0] * small.N for c in other), dtype=np.uint64)
    g.ct_download_many_async(other, back.ctypes.data)
    g.sync()
    assert np.array_equal(back[:2 * 3 * small.N].reshape(2, 3, small.N), g.ct_download(other[0]))
    del batch, other, outs_b


def test_multichannel_special_conv_matches_fp64(conv13):
    """The special conv with C = 2 input channels (Sec. 5.3: tap products over
    both channel blocks, the channel sum by chained rotations of H*W, the A*
    mask, two rescales) decrypts to the FP64 convolution summed over the
    channels."""
    pr = conv13
    g = pr.g
    P = pr.P
    C, H, W, k = 2, 8, 8, 3
    pr.add_keys(OF.conv_rotation_steps(W, k) + [H * W])
    X = synth.image(P["seed"], 40, (C, H, W))
    K = synth.conv_kernel(P["seed"], 41, (1, C, k, k), std=0.3)
    x = np.zeros(pr.N // 2)
    x[:C * H * W] = X.reshape(-1)
    ct = g.encrypt(pr.pk, g.encode(x, pr.L, P["scale"]), nonce=40)
    layer = g.conv2d_prepare(C, k, 1, 1, H, W, K[0], [0.2], pr.L, P["scale"])
    out = g.conv2d_apply(layer, ct)
    assert g.ct_info(out)[0] == pr.L - 2
    y = np.asarray(g.decode(g.decrypt(pr.sk, out))).real
    want = OF.conv2d_fp64(X, K, b=[0.2], pad=1).reshape(-1)
    assert np.max(np.abs(y[:H * W] - want)) < 1e-4
    assert np.max(np.abs(y[H * W:C * H * W])) < 1e-4  # the A* mask cleared the other block
