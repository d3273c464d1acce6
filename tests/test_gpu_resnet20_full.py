"""ResNet-20 at full size on the GPU (N = 2^16, 37 primes, 9 sparse
bootstraps, the ResNet-20 workload's parameters), one CIFAR-shaped
synthetic input:
the decrypted logits against the FP64 network with the same Chebyshev ReLUs
(oracle), within a tolerance derived from the bootstrap's measured precision.

Tolerance.  Apart from the fresh encryption and the layers' key-switching
noise (about 1e-7 of the message at scale 2^40), the encrypted network
differs from the FP64 one by each bootstrap's error: a bootstrap returns its
input (in [-1, 1]: the ReLU's 1/beta is folded into the conv before it) up to
an error d, measured here on a uniform [-1, 1] vector x and split in three
parts: its mean mu over the slots (a shift of every slot alike, carried by
the output's constant coefficient),
a change of scale rho (the least-squares fit d - mu ~ rho x) and a residual
of at most e_r per slot.  The coherent parts are what the layers after a
bootstrap amplify most: a shift of every slot by e_r moves the logits about
fifteen times as far as e_r with random signs.  That error enters the
network at the bootstrapped ReLUs' inputs and is carried to the logits by
the layers after it.  The FP64 network with every bootstrapped ReLU input v
taken to v (1 + s rho) + beta (s mu + e_r r) (s = +1 or -1; r random signs,
slot by slot; beta: the ReLU's bound, the unscaled units of the FP64
network) shows that propagation: A = the largest logit change over both
signs s and four draws of r.  Every slot moved by the full e_r over-states
the residual, so tol = 2 A + 1e-4 bounds the encrypted error with margin.
The distance to the network with exact ReLUs (the Chebyshev approximation's
own error besides) is printed for reference."""
import numpy as np
import pytest

import gpu_common  # noqa: F401  (test set-up module; keeps the import order of the other GPU tests)
from oracle import fheon as OF
from paper_2510_03996_gb300 import resnet as R
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


def bootstrapped_relus(net):
    """Indices of the ReLUs whose input the network bootstraps first."""
    out, r, booted = [], 0, False
    series = set(id(x) for x in net._series.values())
    for op in net.plan:
        if op[0] == "boot":
            booted = True
        elif op[0] == "layer" and id(op[1]) in series:
            if booted:
                out.append(r)
            r += 1
            booted = False
    return out


def test_resnet20_full_size_within_the_bootstrap_tolerance():
    import torch
    from paper_2510_03996_gb300 import fheon as F

    torch.cuda.set_device(0)
    F.use_torch_allocator()
    P = synth.params("resnet_n16")
    N = 1 << P["logN"]
    s = torch.cuda.Stream()
    ctx = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                    stream=s.cuda_stream)
    w = R.weights(P["seed"])
    X = synth.image(P["seed"], 800, (3, 32, 32), dist="normal")
    calib = [X, synth.image(P["seed"], 801, (3, 32, 32), dist="normal")]
    betas = R.relu_bounds(calib, w)
    sk, pk = ctx.keygen()
    net = R.EncryptedResNet(ctx, w, betas, P["scale"])
    assert net.n_boot == 9
    net.keygen(sk)
    ct = ctx.drop_level(ctx.encrypt(pk, ctx.encode(R.pack_input(X, N // 2), ctx.L, P["scale"]), nonce=1),
                        net.in_level)
    y = net.forward(ct)
    assert ctx.ct_info(y)[0] == net.out_level
    logits = np.asarray(ctx.decode(ctx.decrypt(sk, y))).real[:10]

    # the bootstraps' precision on this context (the larger of the sparse one,
    # which returns slots [0, N/4) in both copies, and the full one)
    z = synth.uniform_slots(P["seed"], 802, N // 2)
    zc = ctx.drop_level(ctx.encrypt(pk, ctx.encode(z, ctx.L, P["scale"]), nonce=2), 2)
    rho, mu, e_r = 0.0, 0.0, 0.0
    z0 = z.copy()
    z0[N // 4:] = 0.0       # the unmasked sparse bootstrap's inputs are zero outside its slots
    zc0 = ctx.drop_level(ctx.encrypt(pk, ctx.encode(z0, ctx.L, P["scale"]), nonce=3), 1)
    for (slots, unmasked), layer in net._boots.items():
        v, c = (z0, zc0) if unmasked else (z, zc)
        want_b = np.tile(v[:slots], N // 2 // slots) if slots else v
        d = np.asarray(ctx.decode(ctx.decrypt(sk, ctx.layer_apply(layer, c)))).real - want_b
        m_k = float(np.mean(d))
        r_k = float(np.dot(d - m_k, want_b) / np.dot(want_b, want_b))
        mu = max(mu, abs(m_k))
        rho = max(rho, abs(r_k))
        e_r = max(e_r, float(np.max(np.abs(d - m_k - r_k * want_b))))

    # the oracle's FP64 network with the same Chebyshev ReLUs, and its response
    # to the bootstraps' errors at the bootstrapped ReLUs
    arch = R.FULL
    want = OF.resnet_fp64(X, w, arch["chans"], arch["blocks"], betas=betas)
    booted = set(bootstrapped_relus(net))
    assert len(booted) == 9
    rng = np.random.default_rng(0x7E5)
    A = 0.0
    for sign in (1.0, -1.0):
        for _ in range(4):
            def perturb(i, v):
                if i not in booted:
                    return v
                return v * (1.0 + sign * rho) + betas[i] * (sign * mu + e_r * rng.choice([-1.0, 1.0], size=v.shape))
            A = max(A, float(np.max(np.abs(OF.resnet_fp64(X, w, arch["chans"], arch["blocks"], betas=betas,
                                                          perturb=perturb) - want))))
    tol = 2.0 * A + 1e-4
    err = float(np.max(np.abs(logits - want)))
    exact = OF.resnet_fp64(X, w, arch["chans"], arch["blocks"])
    print("resnet-20 N=2^16: bootstrap mean error %.3g, scale error %.3g, residual %.3g, propagated %.3g, "
          "tolerance %.3g; |enc - fp64 Chebyshev| = %.3g, |enc - fp64 exact ReLU| = %.3g"
          % (mu, rho, e_r, A, tol, err, float(np.max(np.abs(logits - exact)))))
    assert err < tol
    assert int(np.argmax(logits)) == int(np.argmax(want))
    del y, ct, zc, net
    ctx.close()
