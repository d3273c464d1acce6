"""Host-only calls of the library (no device is touched): the ReLU's and
EvalMod's Chebyshev coefficients are the oracle's to the bit (the integer
constants of both sides' series derive from them), the default bootstrapping
parameters follow the oracle's rule, the series depth is the oracle's, and
allocator hooks install and uninstall."""
import numpy as np
import pytest

from oracle import boot as B
from oracle import fheon as OF
from paper_2510_03996_gb300 import fheon as F


@pytest.mark.parametrize("beta,D", [(1.0, 7), (2.5, 27), (4.0, 59), (17.25, 59), (3.0, 127)])
def test_relu_coefficients_identical(beta, D):
    assert np.array_equal(F.relu_coeffs(beta, D), OF.relu_cheb_coeffs(beta, D))


@pytest.mark.parametrize("K,r,D", [(128, 7, 27), (512, 9, 27), (64, 5, 31), (256, 8, 59)])
def test_evalmod_coefficients_identical(K, r, D):
    assert np.array_equal(F.Context.evalmod_coeffs(K, r, D), B.evalmod_coeffs(K, r, D))


def test_series_depths():
    for D in (1, 2, 7, 27, 59, 63, 64, 100, 1023):
        assert F.cheb_depth(D) == OF.cheb_depth(D)
    with pytest.raises(F.FheonError):
        F.cheb_depth(0)


def test_allocator_hooks_install_without_a_gpu():
    """Installing hooks is host-only: a pair installs, NULL/NULL restores
    cudaMalloc, and one hook without the other is refused."""
    from paper_2510_03996_gb300 import fheon as F
    L = F.load()
    F.set_allocator(lambda n, s, u: None, lambda p, n, s, u: None)
    F.set_allocator()
    assert L.fheon_set_allocator(F.ALLOC_FN(lambda n, s, u: None), F.FREE_FN(), None) == -1
    with pytest.raises(F.FheonError):
        F.set_allocator(lambda n, s, u: None)


def test_server_timeout_refuses_a_null_server():
    from paper_2510_03996_gb300 import fheon as F
    assert F.load().fheon_server_set_admit_timeout(None, 1.0) == -1


def test_binding_refuses_arrays_of_the_wrong_size():
    """Sizes the C side would trust are checked before any call: conv kernels
    against the map's channels, FC weights against the map's values, biases
    against the outputs, the one-channel conv's weights."""
    C_ = F.Context
    m = (2, 5, 5, 8, 1, 64)
    K, b = C_._conv_weights(m, np.zeros((3, 2, 3, 3)), [0.1, 0.2, 0.3])
    assert K.shape == (3, 2, 3, 3) and b.size == 3
    for bad_K, bad_b in ((np.zeros((3, 1, 3, 3)), None), (np.zeros((3, 2, 3, 2)), None),
                         (np.zeros((3, 2, 3, 3)), [0.1, 0.2]), (np.zeros((2, 3, 3)), None)):
        with pytest.raises(F.FheonError):
            C_._conv_weights(m, bad_K, bad_b)
    W, b = C_._fc_weights(m, np.zeros((4, 50)), np.zeros(4))
    assert W.shape == (4, 50)
    for bad_W, bad_b in ((np.zeros((4, 49)), None), (np.zeros(50), None), (np.zeros((4, 50)), np.zeros(3))):
        with pytest.raises(F.FheonError):
            C_._fc_weights(m, bad_W, bad_b)
    w, b = C_._conv2d_weights(3, 5, np.zeros((3, 5, 5)), [0.25])
    assert w.size == 75 and b.size == 1
    with pytest.raises(F.FheonError):
        C_._conv2d_weights(3, 5, np.zeros((2, 5, 5)), None)
    with pytest.raises(F.FheonError):
        C_._conv2d_weights(1, 5, np.zeros((5, 5)), [0.1, 0.2])


@pytest.mark.parametrize("k,H,W", [(3, 6, 6), (5, 28, 28), (5, 7, 9)])
def test_special_conv_rotation_steps_are_the_oracle_taps(k, H, W):
    """The special conv's key list: one step per non-identity tap (the oracle's
    list, the same set)."""
    import ctypes
    L = F.load()
    n = ctypes.c_uint32(0)
    pad = (k - 1) // 2
    assert L.fheon_conv2d_rotation_steps(1 << 13, 1, 1, k, 1, pad, H, W, None, ctypes.byref(n)) == 0
    out = (ctypes.c_int32 * n.value)()
    assert L.fheon_conv2d_rotation_steps(1 << 13, 1, 1, k, 1, pad, H, W, out, ctypes.byref(n)) == 0
    want = set(OF.conv_rotation_steps(W, k))
    assert sorted(out) == sorted(want) and len(out) == len(want)
    small = (ctypes.c_int32 * 1)()
    n = ctypes.c_uint32(1)
    assert L.fheon_conv2d_rotation_steps(1 << 13, 1, 1, k, 1, pad, H, W, small, ctypes.byref(n)) == -1  # no room
    assert L.fheon_conv2d_rotation_steps(1000, 1, 1, k, 1, pad, H, W, None, ctypes.byref(n)) == -1  # N not 2^k


@pytest.mark.parametrize("C,Fo,k,s,pad,H", [(3, 4, 3, 2, 1, 8), (2, 3, 5, 1, 0, 12), (16, 16, 3, 1, 1, 32),
                                           (1, 6, 5, 1, 0, 28)])
def test_general_conv_rotation_steps_are_the_oracle_plans(C, Fo, k, s, pad, H):
    """The general conv's key list: the oracle's rotation-sum plan of the
    convolution (taps and block shifts) and, when the outputs are not compact,
    the oracle's repack plan to the compact map."""
    import ctypes
    N = 1 << 16
    n = N // 2
    L = F.load()
    cnt = ctypes.c_uint32(0)
    assert L.fheon_conv2d_rotation_steps(N, C, Fo, k, s, pad, H, H, None, ctypes.byref(cnt)) == 0
    out = (ctypes.c_int32 * cnt.value)()
    assert L.fheon_conv2d_rotation_steps(N, C, Fo, k, s, pad, H, H, out, ctypes.byref(cnt)) == 0
    K = np.ones((Fo, C, k, k))
    r, groups = OF.conv_plan(C, Fo, k, pad, H, H, H, 1, H * H, n, K, stride=s)
    want = set(OF.linear_steps(r, groups))
    Ho = (H + 2 * pad - k) // s + 1
    if s > 1 or Ho != H:
        rr, gg = OF.repack_plan(Fo, Ho, Ho, (H, s, H * H), (Ho, 1, Ho * Ho), n)
        want |= set(OF.linear_steps(rr, gg))
    assert sorted(out) == sorted(want)


def test_context_arguments_refused_before_any_device_work():
    """fheon_ctx_create's documented argument rules (checked on the host, so
    they run without a GPU): N a power of two in [2^10, 2^17], moduli prime,
    = 1 mod 2N, distinct and below 2^60, 1 <= dnum <= nq, digits at most 16."""
    import ctypes
    from oracle import ckks as O
    L = F.load()
    N = 1 << 12
    good = O.gen_primes(N, [50, 50, 50, 60])
    h = ctypes.c_void_p()

    def create(N, q, p, dnum):
        qa = (ctypes.c_uint64 * len(q))(*q)
        pa = (ctypes.c_uint64 * len(p))(*p)
        return L.fheon_ctx_create(N, qa, len(q), pa, len(p), dnum, 2.0 ** 40, 1, None, ctypes.byref(h))

    assert create(N + 1, good[:3], good[3:], 1) == -1                  # not a power of two
    assert create(1 << 9, good[:3], good[3:], 1) == -1                 # below 2^10
    assert create(N, good[:3], good[3:], 4) == -1                      # dnum > nq
    assert create(N, good[:3], good[3:], 0) == -1                      # dnum 0
    assert create(N, [good[0], good[0], good[1]], good[3:], 1) == -1   # repeated modulus
    composite = 3 * 2 * N + 1                                          # 24577 = 7 * 3511, = 1 mod 2N
    assert composite % (2 * N) == 1 and not O.is_prime(composite)
    assert create(N, [good[0], composite], good[3:], 1) == -1          # not prime
    big = O.gen_primes(N, [61])
    assert create(N, good[:2], big, 1) == -1                           # a modulus above 2^60
    assert create(N, [good[0] + 1], good[3:], 1) == -1                 # even, not 1 mod 2N


@pytest.mark.parametrize("name", ["small_n12", "relu_n12", "boot_n12", "conv_n13", "lenet_n15", "rot_n16",
                                  "resnet_n16"])
def test_parameters_picked_on_the_host_are_the_oracles(name):
    """Every parameter set: the library's moduli and NTT roots (host code,
    no device) equal the oracle's, which are written independently."""
    from oracle import ckks as O
    from paper_2510_03996_gb300 import synth
    P = synth.params(name)
    N = 1 << P["logN"]
    bits = P["qbits"] + P["pbits"]
    mods = F.pick_primes(N, bits)
    assert mods == [int(x) for x in O.gen_primes(N, bits)]
    for q in mods[:6] + mods[-2:]:
        assert F.min_root(q, N) == O.min_psi(q, N)


def test_root_and_prime_arguments():
    from oracle import ckks as O
    N = 1 << 12
    q = F.pick_primes(N, [50])[0]
    assert F.min_root(q + 2 * N, N) == 0 or O.is_prime(q + 2 * N)   # not prime: refused, no search
    assert F.min_root(q + 2, N) == 0                                 # not 1 mod 2N
    assert F.min_root(q, N + 1) == 0
    with pytest.raises(F.FheonError):
        F.pick_primes(N + 1, [50])
    with pytest.raises(F.FheonError):
        F.pick_primes(N, [62])


def test_gaussian_table_is_the_oracles():
    from oracle import ckks as O
    assert np.array_equal(F.gaussian_cdt(), np.asarray(O.cdt_table(3.2, 20), dtype=np.uint64))
