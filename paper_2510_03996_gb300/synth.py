"""Seeded synthetic workloads: parameter sets and inputs, no scheme arithmetic.

This module is the only thing the CPU oracle and the CUDA library both see in
a test: it draws message vectors, integer polynomials, images and weights from
numpy's PCG64 with fixed seeds, and it names the parameter sets.  Every random
number the scheme itself draws (keys, encryption noise) comes from each
side's own ChaCha20 stream instead.

Workloads (shapes and distributions of the paper's experiments; MNIST- and
CIFAR-shaped tensors stand in for the datasets, which are not used):
  * conv_n13     - one encrypted 5x5 conv layer, N=2^13, Q={60,40,40} bits,
                   P={60}, dnum=3, scale 2^40, input 1x28x28 ~ U[0,1],
                   kernel ~ N(0, 0.1^2), stride 1, pad 2.
  * rot_n16      - batched rotations, N=2^16, 24 x 50-bit Q + 4 x 60-bit P,
                   dnum=6, 256 ciphertexts at levels ~ U{4..24}, rotation
                   amounts ~ U[1, 2^15).
"""
import numpy as np

SEED_BASE = 0xF4E00000


def params(name):
    """Parameter set by workload name: dict(logN, qbits, pbits, dnum, scale, seed)."""
    if name == "conv_n13":
        return dict(logN=13, qbits=[60, 40, 40], pbits=[60], dnum=3, scale=2.0 ** 40, seed=SEED_BASE + 0)
    if name == "rot_n16":
        return dict(logN=16, qbits=[50] * 24, pbits=[60] * 4, dnum=6, scale=2.0 ** 40, seed=SEED_BASE + 1)
    if name == "tiny":  # test-sized: several limbs, two digits, two P limbs
        return dict(logN=6, qbits=[50, 40, 40, 40], pbits=[58, 58], dnum=2, scale=2.0 ** 30, seed=SEED_BASE + 7)
    if name == "small_n12":  # test-sized, spans several NTT tiles
        return dict(logN=12, qbits=[55, 45, 45, 45, 45], pbits=[60, 60], dnum=3, scale=2.0 ** 40, seed=SEED_BASE + 8)
    if name == "lenet_n15":  # LeNet-5 without bootstrapping: 42 levels of layers + 2 to decrypt from;
        # P (240 bits) above the largest digit (60 + 3 x 40 bits)
        return dict(logN=15, qbits=[60] + [40] * 43, pbits=[60] * 4, dnum=11, scale=2.0 ** 40, seed=SEED_BASE + 2)
    if name == "relu_n12":  # test-sized with the depth of one approximate ReLU (8 levels) and 2 to spare;
        # P (180 bits) above the largest digit (60 + 40 + 40 bits) keeps key-switching noise small
        return dict(logN=12, qbits=[60] + [40] * 10, pbits=[60, 60, 60], dnum=4, scale=2.0 ** 40, seed=SEED_BASE + 9)
    if name == "boot_n12":  # test-sized bootstrapping: q_0 (2^12 above the scale), 2 levels left after it, SlotToCoeff 3 x 50 bits,
        # EvalMod (degree-27 series in 5 levels + 7 doublings) 12 x 60 bits, CoeffToSlot 3 x 60 bits; P 6 x 60 bits
        return dict(logN=12, qbits=[52] + [40] * 2 + [50] * 3 + [60] * 15, pbits=[60] * 6, dnum=4,
                    scale=2.0 ** 40, seed=SEED_BASE + 10)
    if name == "resnet_n16":  # ResNet-20 with bootstrapping: q_0 (2^12 above the scale), 16 levels of layers
        # (two ReLUs and their convolutions between bootstraps), SlotToCoeff 3 x 50 bits, EvalMod (degree-27
        # series in 5 levels + 9 doublings) 14 x 60 bits, CoeffToSlot 3 x 60 bits; P 10 x 60 bits, the size
        # of the largest digit (10 x 60 bits)
        return dict(logN=16, qbits=[52] + [40] * 16 + [50] * 3 + [60] * 17, pbits=[60] * 10, dnum=4,
                    scale=2.0 ** 40, seed=SEED_BASE + 3)
    if name == "resnet_n12":  # test-sized ResNet with bootstrapping: as resnet_n16 with 7 doublings
        return dict(logN=12, qbits=[52] + [40] * 10 + [50] * 3 + [60] * 15, pbits=[60] * 8, dnum=4,
                    scale=2.0 ** 40, seed=SEED_BASE + 11)
    raise KeyError(name)


def rng(seed, stream=0):
    return np.random.Generator(np.random.PCG64([int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)]))


def uniform_slots(seed, stream, n, lo=-1.0, hi=1.0, complex_=False):
    g = rng(seed, stream)
    z = g.uniform(lo, hi, n)
    if complex_:
        z = z + 1j * g.uniform(lo, hi, n)
    return z


def small_int_poly(seed, stream, N, bound):
    """Integer polynomial with coefficients uniform in [-bound, bound]."""
    return rng(seed, stream).integers(-bound, bound + 1, N, dtype=np.int64)


def image(seed, stream, shape, dist="uniform01"):
    g = rng(seed, stream)
    if dist == "uniform01":
        return g.uniform(0.0, 1.0, shape)
    if dist == "normal":
        return g.standard_normal(shape)
    raise KeyError(dist)


def conv_kernel(seed, stream, shape, std=0.1):
    return rng(seed, stream).normal(0.0, std, shape)


def rotation_workload(seed, n_ct=256, lmin=4, lmax=24, rmax=1 << 15):
    """Levels ~ U{lmin..lmax} and rotation amounts ~ U[1, rmax) for n_ct ciphertexts."""
    g = rng(seed, 99)
    levels = g.integers(lmin, lmax + 1, n_ct)
    steps = g.integers(1, rmax, n_ct)
    return [int(x) for x in levels], [int(x) for x in steps]
