"""LeNet-5 encrypted inference end to end on the GPU (N = 2^15, 44 levels,
no bootstrapping): the decrypted logits against the oracle's FP64 LeNet with
the same Chebyshev ReLUs.  The layers themselves are pinned bit-exact against
the oracle at small sizes (test_gpu_layers, test_gpu_relu)."""
import numpy as np
import pytest

from oracle import fheon as OF
from paper_2510_03996_gb300 import lenet, synth

pytestmark = pytest.mark.gpu


def test_lenet_logits_match_fp64():
    import torch
    from paper_2510_03996_gb300 import fheon as F
    torch.cuda.set_device(0)
    F.use_torch_allocator()
    P = synth.params("lenet_n15")
    N = 1 << P["logN"]
    stream = torch.cuda.Stream()  # graph capture needs a created stream
    ctx = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                    stream=stream.cuda_stream)
    w = lenet.weights(P["seed"])
    xs = [synth.image(P["seed"], 600 + s, (1, 28, 28)) for s in range(2)]
    betas = lenet.relu_bounds(xs, w)
    sk, pk = ctx.keygen()
    ctx.relinkeygen(sk)
    net = lenet.EncryptedLeNet(ctx, w, betas, ctx.L, P["scale"])
    ctx.rotkeygen(sk, net.rotation_steps())
    # two convs, two poolings and three FC layers (1 level each), four ReLUs
    assert net.out_level == ctx.L - 7 - sum(lenet.relu_depth(b) for b in betas) and net.out_level >= 2
    for i, X in enumerate(xs):
        ct = ctx.encrypt(pk, ctx.encode(lenet.pack_input(X, N // 2), ctx.L, P["scale"]), nonce=i)
        y = net.forward(ct)
        # the layers replayed as CUDA graphs (captured on the first input) give the same bits
        yg = net.forward_graph(ct)
        assert np.array_equal(ctx.ct_download(yg), ctx.ct_download(y))
        got = np.asarray(ctx.decode(ctx.decrypt(sk, y))).real[:10]
        want = OF.lenet_fp64(X, w, betas)
        assert np.max(np.abs(got - want)) < 1e-2, (got, want)
        exact = OF.lenet_fp64(X, w)
        assert np.max(np.abs(got - exact)) < 0.1
