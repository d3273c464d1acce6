"""Thin Python binding of libfheon (include/fheon.h): the same call names,
argument marshalling only.  Every step runs in the CUDA library; there is no
Python or CPU fallback, and loading fails loudly when the library is missing.

PyTorch provides the device memory (its caching allocator, installed through
``fheon_set_allocator``) and the stream (``torch.cuda.current_stream()``).
"""
import ctypes
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfheon.so")

FHEON_OK = 0
NUM_SCHEDULES = 32  # FHEON_NUM_SCHEDULES
PENDING = 1  # FHEON_PENDING
ERRORS = {-1: "FHEON_ERR_ARG", -2: "FHEON_ERR_OOM", -3: "FHEON_ERR_NO_KEY", -4: "FHEON_ERR_LEVEL",
          -5: "FHEON_ERR_SCALE", -6: "FHEON_ERR_TIMEOUT", -7: "FHEON_ERR_CUDA", -8: "FHEON_ERR_UNIMPLEMENTED"}

c_u32, c_u64, c_i32, c_dbl, c_vp, c_int, c_sz = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t)
P = ctypes.POINTER
c_vpp = P(c_vp)

ALLOC_FN = ctypes.CFUNCTYPE(c_vp, c_sz, c_vp, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, c_sz, c_vp, c_vp)


class fheon_map(ctypes.Structure):
    """Packed layout of a (C, H, W) map: channel c at c*block, (i, j) at + dil*(i*grid + j)."""
    _fields_ = [("C", ctypes.c_uint32), ("H", ctypes.c_uint32), ("W", ctypes.c_uint32),
                ("grid", ctypes.c_uint32), ("dil", ctypes.c_uint32), ("block", ctypes.c_uint32)]

    def tup(self):
        return (self.C, self.H, self.W, self.grid, self.dil, self.block)


class fheon_rot_item(ctypes.Structure):
    _fields_ = [("input", c_vp), ("output", c_vp), ("step", c_i32)]


class fheon_step(ctypes.Structure):
    """One step of a model program (FHEON_STEP_LAYER / _ADD / _SCALE)."""
    _fields_ = [("op", ctypes.c_uint32), ("src", ctypes.c_uint32), ("src2", ctypes.c_uint32),
                ("dst", ctypes.c_uint32), ("level", ctypes.c_uint32), ("layer", c_vp), ("c", ctypes.c_double)]


STEP_LAYER, STEP_ADD, STEP_SCALE = 0, 1, 2


class fheon_boot_params(ctypes.Structure):
    """Bootstrapping: CoeffToSlot / SlotToCoeff levels, EvalMod's range K,
    series degree and double-angle steps, BSGS baby steps (0: fewest rotations),
    message slots (0: all N/2; fewer: the sparse bootstrap), and whether a
    sparse bootstrap's inputs are known to be zero outside those slots (no mask)."""
    _fields_ = [("cts_levels", ctypes.c_uint32), ("stc_levels", ctypes.c_uint32), ("K", ctypes.c_uint32),
                ("degree", ctypes.c_uint32), ("doublings", ctypes.c_uint32), ("baby", ctypes.c_uint32),
                ("slots", ctypes.c_uint32), ("unmasked", ctypes.c_uint32)]


# name -> argument types (all return int unless listed in _RESTYPE)
SIGNATURES = {
    "fheon_error_string": [c_int],
    "fheon_last_error": [c_vp],
    "fheon_set_allocator": [ALLOC_FN, FREE_FN, c_vp],
    "fheon_ctx_create": [c_u32, P(c_u64), c_u32, P(c_u64), c_u32, c_u32, c_dbl, c_u64, c_vp, c_vpp],
    "fheon_ctx_create_bits": [c_u32, P(c_u32), c_u32, P(c_u32), c_u32, c_u32, c_dbl, c_u64, c_vp, c_vpp],
    "fheon_ctx_destroy": [c_vp],
    "fheon_pick_primes": [c_u32, P(c_u32), c_u32, P(c_u64)],
    "fheon_min_root": [c_u64, c_u32],
    "fheon_gaussian_cdt": [P(c_u64), c_u32],
    "fheon_ctx_info": [c_vp, P(c_u32), P(c_u32), P(c_u32), P(c_u32), P(c_u32)],
    "fheon_ctx_moduli": [c_vp, P(c_u64)],
    "fheon_ctx_set_stream": [c_vp, c_vp],
    "fheon_ctx_get_schedule": [c_vp, P(c_int)],
    "fheon_ctx_set_schedule": [c_vp, c_int],
    "fheon_ctx_set_batching": [c_vp, c_int],
    "fheon_autotune_schedule": [c_vp, P(fheon_rot_item), c_u32, c_u32, P(c_int), P(c_dbl)],
    "fheon_sync": [c_vp],
    "fheon_keygen": [c_vp, c_vpp, c_vpp],
    "fheon_sk_destroy": [c_vp],
    "fheon_pk_destroy": [c_vp],
    "fheon_sk_download": [c_vp, c_vp, P(c_u64)],
    "fheon_pk_download": [c_vp, c_vp, P(c_u64)],
    "fheon_rotkeygen": [c_vp, c_vp, P(c_i32), c_u32],
    "fheon_galois_keygen": [c_vp, c_vp, P(c_u64), c_u32],
    "fheon_key_erase": [c_vp, c_u64],
    "fheon_key_stats": [c_vp, P(c_u32), P(c_u64)],
    "fheon_key_download": [c_vp, c_u64, P(c_u64)],
    "fheon_key_upload": [c_vp, c_u64, P(c_u64)],
    "fheon_key_list": [c_vp, P(c_u64), P(c_u32)],
    "fheon_galois_elt": [c_vp, c_i32],
    "fheon_encode_plain": [c_vp, P(c_dbl), P(c_dbl), c_u32, c_u32, c_dbl, c_vpp],
    "fheon_plain_from_coeffs": [c_vp, P(ctypes.c_int64), c_u32, c_dbl, c_vpp],
    "fheon_encode_coeffs": [c_vp, P(c_dbl), P(c_dbl), c_u32, c_dbl, P(ctypes.c_int64)],
    "fheon_decode": [c_vp, c_vp, P(c_dbl), P(c_dbl), c_u32],
    "fheon_pt_info": [c_vp, P(c_u32), P(c_dbl)],
    "fheon_pt_download": [c_vp, c_vp, P(c_u64)],
    "fheon_pt_destroy": [c_vp],
    "fheon_encrypt": [c_vp, c_vp, c_vp, c_vpp],
    "fheon_encrypt_seeded": [c_vp, c_vp, c_vp, c_u64, c_vpp],
    "fheon_decrypt": [c_vp, c_vp, c_vp, c_vpp],
    "fheon_ct_create": [c_vp, c_u32, c_dbl, c_vpp],
    "fheon_ct_destroy": [c_vp],
    "fheon_ct_info": [c_vp, P(c_u32), P(c_dbl)],
    "fheon_ct_upload_async": [c_vp, c_vp, P(c_u64), c_vp],
    "fheon_ct_create_batch": [c_vp, P(c_u32), c_u32, c_dbl, P(c_vp)],
    "fheon_ct_upload_many_async": [c_vp, P(c_vp), c_u32, P(c_u64), c_vp],
    "fheon_ct_download_many_async": [c_vp, P(c_vp), c_u32, P(c_u64), c_vp],
    "fheon_ct_download_async": [c_vp, c_vp, P(c_u64), c_vp],
    "fheon_ct_upload": [c_vp, c_vp, P(c_u64)],
    "fheon_ct_download": [c_vp, c_vp, P(c_u64)],
    "fheon_ct_device_ptr": [c_vp, c_vpp],
    "fheon_rotate": [c_vp, c_vp, c_i32, c_vp],
    "fheon_rotate_galois": [c_vp, c_vp, c_u64, c_vp],
    "fheon_rotate_batch": [c_vp, P(fheon_rot_item), c_u32],
    "fheon_rotate_hoisted": [c_vp, c_vp, P(c_i32), c_u32, P(c_vp)],
    "fheon_rotate_batch_hoisted": [c_vp, P(fheon_rot_item), c_u32],
    "fheon_alu_peak": [c_vp, c_u32, c_u32, c_u32, P(c_dbl)],
    "fheon_layer_plan_info": [c_vp, P(c_u32), P(c_u32), P(c_u32), P(c_u32), P(c_u32)],
    "fheon_layer_plan": [c_vp, P(c_i32), P(c_i32), P(c_i32)],
    "fheon_layer_plain": [c_vp, c_u32, c_u32, c_u32, c_vpp],
    "fheon_layer_sub": [c_vp, c_u32, c_vpp],
    "fheon_layer_coeffs": [c_vp, P(c_dbl), P(c_u32)],
    "fheon_rotate_noalloc": [c_vp, c_vp, c_i32, c_vp],
    "fheon_mul_plain": [c_vp, c_vp, c_vp, c_vp],
    "fheon_mul_relin": [c_vp, c_vp, c_vp, c_vp],
    "fheon_mul_int": [c_vp, c_vp, ctypes.c_int64, c_vp],
    "fheon_add_int": [c_vp, c_vp, ctypes.c_int64, c_vp],
    "fheon_add_const": [c_vp, c_vp, c_dbl, c_vp],
    "fheon_mul_const_rescale": [c_vp, c_vp, c_dbl, c_dbl, c_vp],
    "fheon_relinkeygen": [c_vp, c_vp],
    "fheon_relu_coeffs": [c_dbl, c_u32, P(c_dbl)],
    "fheon_linear_prepare_plain": [c_vp, c_u32, P(c_i32), c_u32, P(c_i32), c_u32, P(c_i32), P(c_vp), c_vp, c_u32,
                                   c_vpp],
    "fheon_fc_prepare_plain": [c_vp, c_u32, P(c_vp), P(c_vp), c_vp, c_u32, c_vpp],
    "fheon_conv_prepare": [c_vp, P(fheon_map), c_u32, c_u32, c_u32, c_u32, P(c_dbl), P(c_dbl), c_u32, c_dbl, c_vpp],
    "fheon_avgpool_prepare": [c_vp, P(fheon_map), c_u32, c_u32, c_u32, c_vpp],
    "fheon_fc_prepare": [c_vp, P(fheon_map), c_u32, P(c_dbl), P(c_dbl), c_u32, c_dbl, c_vpp],
    "fheon_layer_apply": [c_vp, c_vp, c_vp, c_vp],
    "fheon_global_avgpool_prepare": [c_vp, P(fheon_map), c_u32, c_vpp],
    "fheon_repack_prepare": [c_vp, P(fheon_map), P(fheon_map), c_u32, c_vpp],
    "fheon_avgpool": [c_vp, c_vp, P(fheon_map), c_u32, c_u32, c_vp],
    "fheon_global_avgpool": [c_vp, c_vp, P(fheon_map), c_vp],
    "fheon_fc": [c_vp, c_vp, P(fheon_map), c_u32, P(c_dbl), P(c_dbl), c_u32, c_vp],
    "fheon_bootstrap": [c_vp, c_vp, c_vp],
    "fheon_boot_params_default": [c_vp, P(fheon_boot_params)],
    "fheon_evalmod_coeffs": [c_u32, c_u32, c_u32, P(c_dbl)],
    "fheon_bootstrap_prepare": [c_vp, P(fheon_boot_params), c_dbl, c_vpp],
    "fheon_bootstrap_compose": [c_vp, P(fheon_boot_params), P(c_vp), P(c_vp), P(c_dbl), c_dbl, c_vpp],
    "fheon_bootstrap_keygen": [c_vp, c_vp, c_vp],
    "fheon_bootstrap_set_mask": [c_vp, c_vp, c_vp],
    "fheon_bootstrap_info": [c_vp, P(c_u32), P(c_dbl)],
    "fheon_mod_raise": [c_vp, c_vp, c_vp],
    "fheon_selftest_wait": [c_vp, c_u32],
    "fheon_layer_apply_graph": [c_vp, c_vp, c_vp, c_vp],
    "fheon_layer_apply_batch": [c_vp, c_vp, P(c_vp), c_u32, P(c_vp)],
    "fheon_model_create": [c_vp, P(c_vp), c_u32, c_vpp],
    "fheon_model_create_program": [c_vp, P(fheon_step), c_u32, c_u32, c_dbl, c_vpp],
    "fheon_model_run": [c_vp, c_vp, c_vp, c_vp],
    "fheon_model_destroy": [c_vp],
    "fheon_model_footprint": [c_vp, c_u32, P(c_sz)],
    "fheon_server_model_stats": [c_vp, c_vp, P(c_u32), P(c_u64), P(c_sz)],
    "fheon_server_create": [c_vp, c_u32, c_sz, c_vpp],
    "fheon_server_destroy": [c_vp],
    "fheon_server_submit": [c_vp, c_vp, c_vp, P(c_u64)],
    "fheon_server_step": [c_vp, P(c_u32)],
    "fheon_server_result": [c_vp, c_u64, c_vp],
    "fheon_server_set_admit_timeout": [c_vp, c_dbl],
    "fheon_server_set_graphs": [c_vp, c_int],
    "fheon_server_graph_replays": [c_vp, P(c_u64)],
    "fheon_server_stats": [c_vp, P(c_u64), P(c_u32), P(c_u32), P(c_u32)],
    "fheon_layer_rotation_steps": [c_vp, P(c_i32), P(c_u32)],
    "fheon_layer_out_map": [c_vp, P(fheon_map)],
    "fheon_relu_prepare": [c_vp, c_dbl, c_u32, c_u32, c_u32, c_vpp],
    "fheon_relu_prepare_plain": [c_vp, c_dbl, c_u32, c_vp, c_u32, c_vpp],
    "fheon_relu_apply": [c_vp, c_vp, c_vp, c_vp],
    "fheon_cheb_prepare": [c_vp, P(c_dbl), c_u32, c_u32, c_vpp],
    "fheon_cheb_depth": [c_u32],
    "fheon_relu_approx": [c_vp, c_vp, c_dbl, c_u32, c_u32, c_vp],
    "fheon_mac_plain": [c_vp, P(c_vp), P(c_vp), c_u32, c_vp],
    "fheon_add": [c_vp, c_vp, c_vp, c_vp],
    "fheon_add_plain": [c_vp, c_vp, c_vp, c_vp],
    "fheon_rescale": [c_vp, c_vp, c_vp],
    "fheon_drop_level": [c_vp, c_vp, c_u32, c_vp],
    "fheon_conv2d_rotation_steps": [c_u32, c_u32, c_u32, c_u32, c_u32, c_u32, c_u32, c_u32, P(c_i32), P(c_u32)],
    "fheon_conv2d_prepare": [c_vp, c_u32, c_u32, c_u32, c_u32, c_u32, c_u32, P(c_dbl), P(c_dbl), c_u32, c_dbl, c_vpp],
    "fheon_conv2d_prepare_plain": [c_vp, c_u32, c_u32, c_u32, c_u32, c_u32, P(c_vp), c_vp, c_vpp],
    "fheon_conv2d_apply": [c_vp, c_vp, c_vp, c_vp],
    "fheon_conv2d_apply_graph": [c_vp, c_vp, c_vp, c_vp],
    "fheon_conv2d": [c_vp, c_vp, c_u32, c_u32, c_u32, c_u32, c_u32, c_u32, c_u32, P(c_dbl), P(c_dbl), c_vp],
    "fheon_layer_destroy": [c_vp],
    "fheon_profile_begin": [c_vp],
    "fheon_profile_end": [c_vp, ctypes.c_char_p, c_sz],
}
_RESTYPE = {"fheon_error_string": ctypes.c_char_p, "fheon_last_error": ctypes.c_char_p, "fheon_galois_elt": c_u64,
            "fheon_min_root": c_u64,
            "fheon_cheb_depth": c_u32}

_lib = None


def load():
    """Load libfheon.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libfheon.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _RESTYPE.get(name, c_int)
    _lib = L
    return L


def exported_symbols():
    return list(SIGNATURES)


class FheonError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def check(rc, ctx=None):
    if rc != FHEON_OK:
        msg = load().fheon_error_string(rc).decode()
        if ctx:
            last = load().fheon_last_error(ctx).decode()
            # an argument rejected outright leaves the context's message unchanged
            msg = "%s (last message on the context: %s)" % (msg, last) if rc == -1 else last
        raise FheonError(rc, msg)


def __getattr__(name):
    """Module-level access to every C entry point by its own name."""
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)


# ---------------------------------------------------------------- allocator hook
# Every hook pair ever installed stays alive: the library frees each block
# through the pair that allocated it.
_hooks = []
_hook_device = None


def pick_primes(N, bits):
    """The moduli a context of these bit sizes gets (host only)."""
    b = np.ascontiguousarray(bits, dtype=np.uint32)
    out = np.zeros(len(b), dtype=np.uint64)
    check(load().fheon_pick_primes(int(N), b.ctypes.data_as(P(c_u32)), len(b), _u64p(out)))
    return [int(x) for x in out]


def min_root(q, N):
    """The NTT's root for modulus q (0: q is not a prime = 1 mod 2N)."""
    return int(load().fheon_min_root(int(q), int(N)))


def gaussian_cdt():
    out = np.zeros(41, dtype=np.uint64)
    check(load().fheon_gaussian_cdt(_u64p(out), 41))
    return out


def cheb_depth(degree):
    """Levels the library's Chebyshev series of this degree consumes."""
    d = load().fheon_cheb_depth(int(degree))
    if not d:
        raise FheonError(-1, "degree outside [1, 1023]")
    return d


def relu_coeffs(beta, degree=59):
    """Chebyshev coefficients of f(z) = beta * max(0, z) (the library's own)."""
    out = (c_dbl * (degree + 1))()
    check(load().fheon_relu_coeffs(float(beta), degree, out))
    return np.array(out[:])


def set_allocator(alloc=None, free=None):
    """Install Python callables alloc(nbytes, stream, user) -> address or None
    and free(ptr, nbytes, stream, user) as the library's allocator; with
    neither, cudaMalloc/cudaFree.  Blocks made before go back through the hook
    that made them."""
    global _hook_device
    if (alloc is None) != (free is None):
        raise FheonError(-1, "alloc and free come together")
    pair = (ALLOC_FN(alloc), FREE_FN(free)) if alloc is not None else (ALLOC_FN(), FREE_FN())
    _hooks.append(pair)
    check(load().fheon_set_allocator(pair[0], pair[1], None))
    _hook_device = None


def use_torch_allocator():
    """Route every device allocation of the library through torch's caching
    allocator of the current device (a no-op when it is installed already)."""
    global _hook_device
    import torch

    dev = torch.cuda.current_device()
    if _hook_device == dev:
        return

    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0)))
        except Exception:  # out of memory: the C side reports FHEON_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    pair = (ALLOC_FN(_alloc), FREE_FN(_free))
    _hooks.append(pair)
    check(load().fheon_set_allocator(pair[0], pair[1], None))
    _hook_device = dev


# ---------------------------------------------------------------- marshalling helpers
def _u64p(a):
    return a.ctypes.data_as(P(c_u64))


def _need(ok, what):
    """Refuse, before any C call, an array whose size the C side would trust."""
    if not ok:
        raise FheonError(-1, what)


def _bias(bias, n):
    if bias is None:
        return None
    b = np.ascontiguousarray(bias, dtype=np.float64).reshape(-1)
    _need(b.size == n, "bias needs %d values, got %d" % (n, b.size))
    return b


def _dblp(a):
    return a.ctypes.data_as(P(c_dbl)) if a is not None else None


class Context:
    """Owning wrapper of a fheon_ctx* with one method per C call (marshalling only)."""

    def __init__(self, N, q=None, p=None, dnum=1, scale=2.0 ** 40, seed=0, stream=None, qbits=None, pbits=None):
        L = load()
        h = c_vp()
        st = c_vp(stream) if stream else None
        if qbits is not None:
            qb = np.ascontiguousarray(qbits, dtype=np.uint32)
            pb = np.ascontiguousarray(pbits, dtype=np.uint32)
            rc = L.fheon_ctx_create_bits(N, qb.ctypes.data_as(P(c_u32)), len(qb), pb.ctypes.data_as(P(c_u32)),
                                         len(pb), dnum, scale, seed, st, ctypes.byref(h))
        else:
            qa = np.ascontiguousarray(q, dtype=np.uint64)
            pa = np.ascontiguousarray(p, dtype=np.uint64)
            rc = L.fheon_ctx_create(N, _u64p(qa), len(qa), _u64p(pa), len(pa), dnum, scale, seed, st,
                                    ctypes.byref(h))
        check(rc)
        self.h = h
        info = [c_u32() for _ in range(5)]
        check(L.fheon_ctx_info(h, *[ctypes.byref(x) for x in info]), h)
        self.N, self.L, self.K, self.alpha, self.beta = [x.value for x in info]
        mods = np.zeros(self.L + self.K, dtype=np.uint64)
        check(L.fheon_ctx_moduli(h, _u64p(mods)), h)
        self.moduli = [int(x) for x in mods]
        self.scale = scale

    def close(self):
        if self.h:
            load().fheon_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit torch's allocator may already be torn down: leak instead
        if sys is None or sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        check(rc, self.h)

    # streams
    def set_stream(self, stream):
        self._chk(load().fheon_ctx_set_stream(self.h, c_vp(stream) if stream else None))

    def sync(self):
        self._chk(load().fheon_sync(self.h))

    def get_schedule(self):
        s = c_int()
        self._chk(load().fheon_ctx_get_schedule(self.h, ctypes.byref(s)))
        return s.value

    def set_schedule(self, schedule):
        self._chk(load().fheon_ctx_set_schedule(self.h, int(schedule)))

    def set_batching(self, on):
        """False: the plain one-ciphertext-per-launch path (fheon_ctx_set_batching)."""
        self._chk(load().fheon_ctx_set_batching(self.h, 1 if on else 0))

    def autotune_schedule(self, ins, outs, steps, reps=2, cache=None):
        """Time every allowed key-switching schedule on this batch; keep the fastest.
        Returns (best, {schedule: ms per batch}).  With `cache` (a JSON file
        path), a choice made before for the same parameters and batch shape
        (count and levels) is reused without timing, and new choices are saved."""
        key = None
        if cache is not None:
            import json
            levels = sorted(self.ct_info(c)[0] for c in ins)
            key = "N%d_L%d_K%d_a%d_n%d_l%s" % (self.N, self.L, self.K, self.alpha, len(ins),
                                              ",".join(str(x) for x in levels))
            try:
                with open(cache) as f:
                    known = json.load(f)
            except (OSError, ValueError):
                known = {}
            if key in known:
                self.set_schedule(int(known[key]["schedule"]))
                return int(known[key]["schedule"]), {int(k): v for k, v in known[key]["ms"].items()}
        best, ms = self._autotune(ins, outs, steps, reps)
        if key is not None:
            known[key] = {"schedule": best, "ms": {str(k): v for k, v in ms.items()}}
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(known, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return best, ms

    def _autotune(self, ins, outs, steps, reps):
        items = (fheon_rot_item * len(ins))()
        for i, (a, b, s) in enumerate(zip(ins, outs, steps)):
            items[i].input, items[i].output, items[i].step = a.h, b.h, int(s)
        best = c_int()
        ms = (c_dbl * NUM_SCHEDULES)()
        self._chk(load().fheon_autotune_schedule(self.h, items, len(ins), reps, ctypes.byref(best), ms))
        return best.value, {s: ms[s] for s in range(NUM_SCHEDULES) if ms[s] >= 0}

    # keys
    def keygen(self):
        sk, pk = c_vp(), c_vp()
        self._chk(load().fheon_keygen(self.h, ctypes.byref(sk), ctypes.byref(pk)))
        return Handle(sk, load().fheon_sk_destroy), Handle(pk, load().fheon_pk_destroy)

    def sk_download(self, sk):
        out = np.zeros((self.L + self.K, self.N), dtype=np.uint64)
        self._chk(load().fheon_sk_download(self.h, sk.h, _u64p(out)))
        return out

    def pk_download(self, pk):
        out = np.zeros((2, self.L, self.N), dtype=np.uint64)
        self._chk(load().fheon_pk_download(self.h, pk.h, _u64p(out)))
        return out

    def rotkeygen(self, sk, steps):
        a = np.ascontiguousarray(steps, dtype=np.int32)
        self._chk(load().fheon_rotkeygen(self.h, sk.h, a.ctypes.data_as(P(c_i32)), len(a)))

    def galois_keygen(self, sk, gs):
        a = np.ascontiguousarray(gs, dtype=np.uint64)
        self._chk(load().fheon_galois_keygen(self.h, sk.h, _u64p(a), len(a)))

    def key_erase(self, g):
        self._chk(load().fheon_key_erase(self.h, int(g)))

    def key_stats(self):
        n, b = c_u32(), c_u64()
        self._chk(load().fheon_key_stats(self.h, ctypes.byref(n), ctypes.byref(b)))
        return n.value, b.value

    def key_download(self, g):
        out = np.zeros((self.beta, 2, self.L + self.K, self.N), dtype=np.uint64)
        self._chk(load().fheon_key_download(self.h, int(g), _u64p(out)))
        return out

    def key_upload(self, g, limbs):
        a = np.ascontiguousarray(limbs, dtype=np.uint64)
        if a.size != self.beta * 2 * (self.L + self.K) * self.N:
            raise FheonError(-1, "key limbs must be u64[beta][2][L+K][N]")
        self._chk(load().fheon_key_upload(self.h, int(g), _u64p(a)))

    def key_list(self):
        n = c_u32()
        self._chk(load().fheon_key_list(self.h, None, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1), dtype=np.uint64)
        self._chk(load().fheon_key_list(self.h, _u64p(out), ctypes.byref(n)))
        return [int(x) for x in out[:n.value]]

    def galois_elt(self, r):
        return int(load().fheon_galois_elt(self.h, int(r)))

    # plaintexts
    def plain_from_coeffs(self, coeffs, level, scale=1.0):
        c = np.ascontiguousarray(coeffs, dtype=np.int64)
        _need(c.size == self.N, "plain_from_coeffs needs N = %d coefficients, got %d" % (self.N, c.size))
        h = c_vp()
        self._chk(load().fheon_plain_from_coeffs(self.h, c.ctypes.data_as(P(ctypes.c_int64)), level, scale,
                                                 ctypes.byref(h)))
        return Handle(h, load().fheon_pt_destroy)

    def encode(self, z, level, scale):
        z = np.asarray(z, dtype=np.complex128)
        re, im = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        h = c_vp()
        self._chk(load().fheon_encode_plain(self.h, _dblp(re), _dblp(im), len(z), level, scale, ctypes.byref(h)))
        return Handle(h, load().fheon_pt_destroy)

    def encode_coeffs(self, z, scale):
        z = np.asarray(z, dtype=np.complex128)
        re, im = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        out = np.zeros(self.N, dtype=np.int64)
        self._chk(load().fheon_encode_coeffs(self.h, _dblp(re), _dblp(im), len(z), scale,
                                             out.ctypes.data_as(P(ctypes.c_int64))))
        return out

    def decode(self, pt, n=None):
        n = n or self.N // 2
        re, im = np.zeros(n), np.zeros(n)
        self._chk(load().fheon_decode(self.h, pt.h, _dblp(re), _dblp(im), n))
        return re + 1j * im

    def pt_download(self, pt):
        lv = c_u32()
        check(load().fheon_pt_info(pt.h, ctypes.byref(lv), None))
        out = np.zeros((lv.value, self.N), dtype=np.uint64)
        self._chk(load().fheon_pt_download(self.h, pt.h, _u64p(out)))
        return out

    # ciphertexts
    def encrypt(self, pk, pt, nonce=None):
        h = c_vp()
        if nonce is None:
            self._chk(load().fheon_encrypt(self.h, pk.h, pt.h, ctypes.byref(h)))
        else:
            self._chk(load().fheon_encrypt_seeded(self.h, pk.h, pt.h, int(nonce), ctypes.byref(h)))
        return Handle(h, load().fheon_ct_destroy)

    def decrypt(self, sk, ct):
        h = c_vp()
        self._chk(load().fheon_decrypt(self.h, sk.h, ct.h, ctypes.byref(h)))
        return Handle(h, load().fheon_pt_destroy)

    def ct_create(self, level, scale=1.0):
        h = c_vp()
        self._chk(load().fheon_ct_create(self.h, level, scale, ctypes.byref(h)))
        return Handle(h, load().fheon_ct_destroy)

    def pt_info(self, pt):
        lv, sc = c_u32(), c_dbl()
        check(load().fheon_pt_info(pt.h, ctypes.byref(lv), ctypes.byref(sc)))
        return lv.value, sc.value

    def ct_info(self, ct):
        lv, sc = c_u32(), c_dbl()
        check(load().fheon_ct_info(ct.h, ctypes.byref(lv), ctypes.byref(sc)))
        return lv.value, sc.value

    def ct_upload(self, ct, host):
        host = np.ascontiguousarray(host, dtype=np.uint64)
        level = self.ct_info(ct)[0]
        _need(host.size == 2 * level * self.N, "ct_upload needs u64[2][%d][%d]" % (level, self.N))
        self._chk(load().fheon_ct_upload(self.h, ct.h, _u64p(host)))
        return host  # keep alive until synchronised when pinned/asynchronous

    def ct_upload_ptr(self, ct, host_ptr):
        self._chk(load().fheon_ct_upload(self.h, ct.h, ctypes.cast(c_vp(host_ptr), P(c_u64))))

    def ct_download(self, ct):
        lv, _ = self.ct_info(ct)
        out = np.zeros((2, lv, self.N), dtype=np.uint64)
        self._chk(load().fheon_ct_download(self.h, ct.h, _u64p(out)))
        return out

    def ct_create_batch(self, levels, scale=1.0):
        n = len(levels)
        lv = (c_u32 * n)(*[int(x) for x in levels])
        hs = (c_vp * n)()
        self._chk(load().fheon_ct_create_batch(self.h, lv, n, float(scale), hs))
        return [Handle(c_vp(hs[i]), load().fheon_ct_destroy) for i in range(n)]

    def ct_upload_many_async(self, cts, host_ptr, stream=None):
        arr = (c_vp * len(cts))(*[c.h.value for c in cts])
        self._chk(load().fheon_ct_upload_many_async(self.h, arr, len(cts), ctypes.cast(c_vp(host_ptr), P(c_u64)),
                                                    stream))

    def ct_download_many_async(self, cts, host_ptr, stream=None):
        arr = (c_vp * len(cts))(*[c.h.value for c in cts])
        self._chk(load().fheon_ct_download_many_async(self.h, arr, len(cts), ctypes.cast(c_vp(host_ptr), P(c_u64)),
                                                      stream))

    def ct_upload_async(self, ct, host_ptr, stream=None):
        self._chk(load().fheon_ct_upload_async(self.h, ct.h, ctypes.cast(c_vp(host_ptr), P(c_u64)), stream))

    def ct_download_async(self, ct, host_ptr, stream=None):
        self._chk(load().fheon_ct_download_async(self.h, ct.h, ctypes.cast(c_vp(host_ptr), P(c_u64)), stream))

    def ct_download_ptr(self, ct, host_ptr):
        self._chk(load().fheon_ct_download(self.h, ct.h, ctypes.cast(c_vp(host_ptr), P(c_u64))))

    def ct_device_ptr(self, ct):
        p = c_vp()
        check(load().fheon_ct_device_ptr(ct.h, ctypes.byref(p)))
        return p.value

    # evaluation
    def rotate(self, ct, step, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_rotate(self.h, ct.h, int(step), out.h))
        return out

    def rotate_galois(self, ct, g, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_rotate_galois(self.h, ct.h, int(g), out.h))
        return out

    def rotate_noalloc(self, ct, step, out):
        """Rotation into a caller-made output, with the library's fixed scratch (no allocation)."""
        self._chk(load().fheon_rotate_noalloc(self.h, ct.h, int(step), out.h))
        return out

    @staticmethod
    def _items(ins, outs, steps):
        items = (fheon_rot_item * len(ins))()
        for i, (a, b, s) in enumerate(zip(ins, outs, steps)):
            items[i].input, items[i].output, items[i].step = a.h, b.h, int(s)
        return items

    def rotate_batch(self, ins, outs, steps):
        self._chk(load().fheon_rotate_batch(self.h, self._items(ins, outs, steps), len(ins)))

    def rotate_hoisted(self, ct, steps, outs=None):
        """Rotations of one ciphertext by every step, sharing one raising of c1."""
        outs = outs or [self.ct_create(1) for _ in steps]
        st = (c_i32 * len(steps))(*[int(x) for x in steps])
        hs = (c_vp * len(steps))(*[o.h for o in outs])
        self._chk(load().fheon_rotate_hoisted(self.h, ct.h, st, len(steps), hs))
        return outs

    def rotate_batch_hoisted(self, ins, outs, steps):
        self._chk(load().fheon_rotate_batch_hoisted(self.h, self._items(ins, outs, steps), len(ins)))

    def mul_plain(self, ct, pt, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_mul_plain(self.h, ct.h, pt.h, out.h))
        return out

    def relinkeygen(self, sk):
        self._chk(load().fheon_relinkeygen(self.h, sk.h))

    def mul_relin(self, a, b, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_mul_relin(self.h, a.h, b.h, out.h))
        return out

    def mul_int(self, ct, v, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_mul_int(self.h, ct.h, int(v), out.h))
        return out

    def add_int(self, ct, v, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_add_int(self.h, ct.h, int(v), out.h))
        return out

    def add_const(self, ct, c, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_add_const(self.h, ct.h, float(c), out.h))
        return out

    def mul_const_rescale(self, ct, c, target, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_mul_const_rescale(self.h, ct.h, float(c), float(target), out.h))
        return out

    @staticmethod
    def _map(m):
        return m if isinstance(m, fheon_map) else fheon_map(*[int(x) for x in m])

    def linear_prepare_plain(self, r, s, pts, level, bias=None, fold=()):
        """pts: [len(s)][len(r)] plaintexts or None."""
        nt, ng, nf = len(r), len(s), len(fold)
        rr = (c_i32 * nt)(*[int(x) for x in r])
        ss = (c_i32 * ng)(*[int(x) for x in s])
        ff = (c_i32 * max(1, nf))(*[int(x) for x in fold])
        pp = (c_vp * (nt * ng))(*[(p.h.value if p is not None else None) for row in pts for p in row])
        h = c_vp()
        self._chk(load().fheon_linear_prepare_plain(self.h, nf, ff if nf else None, nt, rr, ng, ss, pp,
                                                    bias.h if bias is not None else None, level, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def fc_prepare_plain(self, W, E, level, bias=None):
        m = len(W)
        ww = (c_vp * m)(*[p.h.value for p in W])
        ee = (c_vp * m)(*[p.h.value for p in E])
        h = c_vp()
        self._chk(load().fheon_fc_prepare_plain(self.h, m, ww, ee, bias.h if bias is not None else None, level,
                                                ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def conv_prepare(self, in_map, K, pad, level, in_scale, bias=None, stride=1):
        K, b = self._conv_weights(in_map, K, bias)
        F, C, k, _ = K.shape
        h = c_vp()
        self._chk(load().fheon_conv_prepare(self.h, ctypes.byref(self._map(in_map)), F, k, stride, pad, _dblp(K),
                                            _dblp(b) if b is not None else None, level, float(in_scale),
                                            ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def avgpool_prepare(self, in_map, k, stride, level):
        h = c_vp()
        self._chk(load().fheon_avgpool_prepare(self.h, ctypes.byref(self._map(in_map)), k, stride, level,
                                               ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    @staticmethod
    def _conv_weights(in_map, K, bias):
        K = np.ascontiguousarray(K, dtype=np.float64)
        m = Context._map(in_map)
        _need(K.ndim == 4 and K.shape[1] == m.C and K.shape[2] == K.shape[3],
              "conv kernel must be K[F][%d][k][k], got shape %s" % (m.C, K.shape))
        return K, _bias(bias, K.shape[0])

    @staticmethod
    def _fc_weights(in_map, W, bias):
        W = np.ascontiguousarray(W, dtype=np.float64)
        m = Context._map(in_map)
        _need(W.ndim == 2 and W.shape[1] == m.C * m.H * m.W,
              "FC weights must be W[m][%d], got shape %s" % (m.C * m.H * m.W, W.shape))
        return W, _bias(bias, W.shape[0])

    def fc_prepare(self, in_map, W, level, in_scale, bias=None):
        W, b = self._fc_weights(in_map, W, bias)
        h = c_vp()
        self._chk(load().fheon_fc_prepare(self.h, ctypes.byref(self._map(in_map)), W.shape[0], _dblp(W),
                                          _dblp(b) if b is not None else None, level, float(in_scale),
                                          ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def repack_prepare(self, in_map, out_map, level):
        h = c_vp()
        self._chk(load().fheon_repack_prepare(self.h, ctypes.byref(self._map(in_map)), ctypes.byref(self._map(out_map)),
                                              level, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def global_avgpool_prepare(self, in_map, level):
        h = c_vp()
        self._chk(load().fheon_global_avgpool_prepare(self.h, ctypes.byref(self._map(in_map)), level, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def avgpool(self, ct, in_map, k, stride, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_avgpool(self.h, ct.h, ctypes.byref(self._map(in_map)), k, stride, out.h))
        return out

    def global_avgpool(self, ct, in_map, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_global_avgpool(self.h, ct.h, ctypes.byref(self._map(in_map)), out.h))
        return out

    def fc(self, ct, in_map, W, bias=None, max_keys=0, out=None):
        W, b = self._fc_weights(in_map, W, bias)
        out = out or self.ct_create(1)
        self._chk(load().fheon_fc(self.h, ct.h, ctypes.byref(self._map(in_map)), W.shape[0], _dblp(W),
                                  _dblp(b) if b is not None else None, max_keys, out.h))
        return out

    def bootstrap(self, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_bootstrap(self.h, ct.h, out.h))
        return out

    def boot_params_default(self):
        p = fheon_boot_params()
        self._chk(load().fheon_boot_params_default(self.h, ctypes.byref(p)))
        return p

    @staticmethod
    def evalmod_coeffs(K, doublings, degree):
        out = (c_dbl * (degree + 1))()
        check(load().fheon_evalmod_coeffs(K, doublings, degree, out))
        return np.array(out[:], dtype=np.float64)

    def bootstrap_prepare(self, in_scale, params=None):
        h = c_vp()
        self._chk(load().fheon_bootstrap_prepare(self.h, ctypes.byref(params) if params is not None else None,
                                                 float(in_scale), ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def bootstrap_compose(self, params, cts, stc, coeffs, in_scale):
        """cts / stc: prepared rotation-sum layers (kept alive by the result)."""
        c = (c_vp * len(cts))(*[x.h.value for x in cts])
        t = (c_vp * len(stc))(*[x.h.value for x in stc])
        cf = np.ascontiguousarray(coeffs, dtype=np.float64)
        _need(cf.size == params.degree + 1, "EvalMod needs degree + 1 = %d coefficients" % (params.degree + 1))
        h = c_vp()
        self._chk(load().fheon_bootstrap_compose(self.h, ctypes.byref(params), c, t, _dblp(cf), float(in_scale),
                                                 ctypes.byref(h)))
        out = Handle(h, load().fheon_layer_destroy)
        out.levels = list(cts) + list(stc)
        return out

    def bootstrap_keygen(self, sk, layer):
        self._chk(load().fheon_bootstrap_keygen(self.h, sk.h, layer.h))

    def bootstrap_set_mask(self, layer, mask):
        """Sparse bootstrap: use the plaintext `mask` (kept alive by the layer)
        as the input mask."""
        self._chk(load().fheon_bootstrap_set_mask(self.h, layer.h, mask.h))
        layer.mask_ref = mask

    @staticmethod
    def bootstrap_info(layer):
        lv, sc = c_u32(0), c_dbl(0)
        check(load().fheon_bootstrap_info(layer.h, ctypes.byref(lv), ctypes.byref(sc)))
        return lv.value, sc.value

    def selftest_wait(self, polls):
        """Launch a bounded wait that runs out (see fheon_selftest_wait)."""
        self._chk(load().fheon_selftest_wait(self.h, polls))

    def mod_raise(self, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_mod_raise(self.h, ct.h, out.h))
        return out

    def layer_apply(self, layer, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_layer_apply(self.h, layer.h, ct.h, out.h))
        return out

    def layer_apply_graph(self, layer, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_layer_apply_graph(self.h, layer.h, ct.h, out.h))
        return out

    def layer_apply_batch(self, layer, cts, outs=None):
        outs = outs or [self.ct_create(1) for _ in cts]
        n = len(cts)
        ii = (c_vp * n)(*[c.h.value for c in cts])
        oo = (c_vp * n)(*[o.h.value for o in outs])
        self._chk(load().fheon_layer_apply_batch(self.h, layer.h, ii, n, oo))
        return outs

    def model(self, layers):
        n = len(layers)
        arr = (c_vp * n)(*[x.h.value for x in layers])
        h = c_vp()
        self._chk(load().fheon_model_create(self.h, arr, n, ctypes.byref(h)))
        m = Handle(h, load().fheon_model_destroy)
        m.layers = list(layers)  # the layers outlive the model
        return m

    def model_program(self, steps, nreg, scale):
        """steps: (op, src, src2, dst, level, layer or None, c) tuples."""
        n = len(steps)
        arr = (fheon_step * n)()
        for i, (op, a, b, d, lv, layer, c) in enumerate(steps):
            arr[i] = fheon_step(op, a, b, d, lv, layer.h.value if layer is not None else None, float(c))
        h = c_vp()
        self._chk(load().fheon_model_create_program(self.h, arr, n, nreg, float(scale), ctypes.byref(h)))
        m = Handle(h, load().fheon_model_destroy)
        m.layers = [st[5] for st in steps if st[5] is not None]  # the layers outlive the model
        return m

    def model_run(self, model, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_model_run(self.h, model.h, ct.h, out.h))
        return out

    def server(self, max_active, mem_budget=0):
        """A server (fheon_server_create); it takes models of other contexts too."""
        h = c_vp()
        self._chk(load().fheon_server_create(self.h, max_active, int(mem_budget), ctypes.byref(h)))
        return Server(self, Handle(h, load().fheon_server_destroy))

    @staticmethod
    def model_footprint(model, level):
        b = c_sz(0)
        check(load().fheon_model_footprint(model.h, level, ctypes.byref(b)))
        return b.value

    @staticmethod
    def layer_rotation_steps(layer):
        n = c_u32(0)
        check(load().fheon_layer_rotation_steps(layer.h, None, ctypes.byref(n)))
        out = (c_i32 * max(1, n.value))()
        check(load().fheon_layer_rotation_steps(layer.h, out, ctypes.byref(n)))
        return list(out[:n.value])

    PLAIN = {"product": 0, "place": 1, "bias": 2, "mask": 3, "mono": 4, "boot_mask": 5}

    @staticmethod
    def layer_plan(layer):
        """{'kind', 'level', 'fold', 'r', 's'} of a prepared layer (fold/r/s for
        rotation-sum layers; counts only otherwise)."""
        v = [c_u32(0) for _ in range(5)]
        check(load().fheon_layer_plan_info(layer.h, *[ctypes.byref(x) for x in v]))
        kind, level, nf, nt, ng = [x.value for x in v]
        out = {"kind": kind, "level": level, "nf": nf, "nt": nt, "ng": ng}
        if kind == 2:
            f, r, s = (c_i32 * max(1, nf))(), (c_i32 * max(1, nt))(), (c_i32 * max(1, ng))()
            check(load().fheon_layer_plan(layer.h, f, r, s))
            out.update(fold=list(f[:nf]), r=list(r[:nt]), s=list(s[:ng]))
        return out

    @staticmethod
    def layer_plain(layer, which, g=0, t=0):
        """A borrowed plaintext of the layer (None where it has none); it keeps
        the layer alive."""
        h = c_vp()
        check(load().fheon_layer_plain(layer.h, Context.PLAIN[which], g, t, ctypes.byref(h)))
        if not h.value:
            return None
        pt = Handle(h, lambda _h: None)
        pt.owner = layer
        return pt

    @staticmethod
    def layer_sub(layer, i):
        """Level i of a bootstrap layer (borrowed; keeps the bootstrap alive)."""
        h = c_vp()
        check(load().fheon_layer_sub(layer.h, i, ctypes.byref(h)))
        sub = Handle(h, lambda _h: None)
        sub.owner = layer
        return sub

    @staticmethod
    def layer_coeffs(layer):
        n = c_u32(0)
        check(load().fheon_layer_coeffs(layer.h, None, ctypes.byref(n)))
        out = (c_dbl * max(1, n.value))()
        check(load().fheon_layer_coeffs(layer.h, out, ctypes.byref(n)))
        return np.array(out[:n.value])

    @staticmethod
    def layer_out_map(layer):
        m = fheon_map()
        check(load().fheon_layer_out_map(layer.h, ctypes.byref(m)))
        return m.tup()

    def relu_prepare(self, beta, degree, n, level):
        h = c_vp()
        self._chk(load().fheon_relu_prepare(self.h, float(beta), degree, n, level, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def relu_prepare_plain(self, beta, degree, mask, level):
        h = c_vp()
        self._chk(load().fheon_relu_prepare_plain(self.h, float(beta), degree, mask.h if mask is not None else None,
                                                  level, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def cheb_prepare(self, coeffs, level):
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        h = c_vp()
        self._chk(load().fheon_cheb_prepare(self.h, _dblp(c), len(c) - 1, level, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def relu_apply(self, layer, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_relu_apply(self.h, layer.h, ct.h, out.h))
        return out

    def relu_approx(self, ct, beta, degree=59, n=None, out=None):
        out = out or self.ct_create(1)
        n = self.N // 2 if n is None else n
        self._chk(load().fheon_relu_approx(self.h, ct.h, float(beta), degree, n, out.h))
        return out

    def mac_plain(self, cts, pts, out=None):
        """out = sum_t cts[t] * pts[t] in one pass."""
        out = out or self.ct_create(1)
        n = len(cts)
        ch = (c_vp * n)(*[c.h for c in cts])
        ph = (c_vp * n)(*[p.h for p in pts])
        self._chk(load().fheon_mac_plain(self.h, ch, ph, n, out.h))
        return out

    def add(self, a, b, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_add(self.h, a.h, b.h, out.h))
        return out

    def add_plain(self, ct, pt, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_add_plain(self.h, ct.h, pt.h, out.h))
        return out

    def rescale(self, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_rescale(self.h, ct.h, out.h))
        return out

    def drop_level(self, ct, level, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_drop_level(self.h, ct.h, level, out.h))
        return out

    # instrumentation
    def profile_begin(self):
        self._chk(load().fheon_profile_begin(self.h))

    def profile_end(self):
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._chk(load().fheon_profile_end(self.h, buf, len(buf)))
        return {k: (v[0], v[1]) for k, v in json.loads(buf.value.decode()).items()}

    PEAK_KINDS = {"ct_lazy": 0, "gs_lazy": 1, "ct_harvey": 2, "gs_harvey": 3, "mac": 4}

    def alu_peak(self, kind, rounds=2048, reps=5):
        """Measured rate (steps/s) of one modular step (see fheon_alu_peak):
        kind is one of PEAK_KINDS."""
        v = c_dbl(0.0)
        self._chk(load().fheon_alu_peak(self.h, self.PEAK_KINDS[kind], rounds, reps, ctypes.byref(v)))
        return v.value

    # layers
    def conv2d_rotation_steps(self, in_ch, out_ch, k, stride, pad, in_h, in_w):
        """Rotation keys fheon_conv2d needs for this shape on this ring."""
        n = c_u32(0)
        check(load().fheon_conv2d_rotation_steps(self.N, in_ch, out_ch, k, stride, pad, in_h, in_w, None,
                                                 ctypes.byref(n)))
        out = np.zeros(max(1, n.value), dtype=np.int32)
        check(load().fheon_conv2d_rotation_steps(self.N, in_ch, out_ch, k, stride, pad, in_h, in_w,
                                                 out.ctypes.data_as(P(c_i32)), ctypes.byref(n)))
        return [int(x) for x in out[:n.value]]

    @staticmethod
    def _conv2d_weights(in_ch, k, w, bias):
        w = np.ascontiguousarray(w, dtype=np.float64)
        _need(w.size == in_ch * k * k, "conv2d weights must be w[%d][%d][%d]" % (in_ch, k, k))
        return w, _bias(bias, 1)

    def conv2d_prepare(self, in_ch, k, stride, pad, in_h, in_w, w, bias, level, in_scale):
        w, b = self._conv2d_weights(in_ch, k, w, bias)
        h = c_vp()
        self._chk(load().fheon_conv2d_prepare(self.h, in_ch, k, stride, pad, in_h, in_w, _dblp(w), _dblp(b), level,
                                              in_scale, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def conv2d_prepare_plain(self, in_ch, k, in_h, in_w, level, taps, bias=None):
        arr = (c_vp * len(taps))(*[t.h for t in taps])
        h = c_vp()
        self._chk(load().fheon_conv2d_prepare_plain(self.h, in_ch, k, in_h, in_w, level, arr,
                                                    bias.h if bias is not None else None, ctypes.byref(h)))
        return Handle(h, load().fheon_layer_destroy)

    def conv2d_apply(self, layer, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_conv2d_apply(self.h, layer.h, ct.h, out.h))
        return out

    def conv2d_apply_graph(self, layer, ct, out=None):
        out = out or self.ct_create(1)
        self._chk(load().fheon_conv2d_apply_graph(self.h, layer.h, ct.h, out.h))
        return out

    def conv2d(self, ct, in_ch, out_ch, k, stride, pad, in_h, in_w, w, bias=None, out=None):
        """w: w[out_ch][in_ch][k][k]; bias: out_ch values or None (fheon_conv2d)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        _need(w.size == out_ch * in_ch * k * k,
              "conv2d weights must be w[%d][%d][%d][%d], got %d values" % (out_ch, in_ch, k, k, w.size))
        b = _bias(bias, out_ch)
        out = out or self.ct_create(1)
        self._chk(load().fheon_conv2d(self.h, ct.h, in_ch, out_ch, k, stride, pad, in_h, in_w, _dblp(w), _dblp(b),
                                      out.h))
        return out


class Server:
    """Continuous-batching server (fheon_server_*)."""

    def __init__(self, ctx, handle):
        self.ctx, self.handle = ctx, handle
        self.models = []

    def submit(self, model, ct):
        rid = c_u64()
        self.ctx._chk(load().fheon_server_submit(self.handle.h, model.h, ct.h, ctypes.byref(rid)))
        self.models.append(model)
        return rid.value

    def step(self):
        n = c_u32()
        self.ctx._chk(load().fheon_server_step(self.handle.h, ctypes.byref(n)))
        return n.value

    def result(self, rid, out=None):
        """The result ciphertext, or None while the request runs."""
        out = out or self.ctx.ct_create(1)
        rc = load().fheon_server_result(self.handle.h, rid, out.h)
        if rc == PENDING:
            return None
        self.ctx._chk(rc)
        return out

    def set_admit_timeout(self, seconds):
        self.ctx._chk(load().fheon_server_set_admit_timeout(self.handle.h, float(seconds)))

    def set_graphs(self, on=True):
        """Single-request layer steps as replayed CUDA graphs on pooled buffers."""
        self.ctx._chk(load().fheon_server_set_graphs(self.handle.h, 1 if on else 0))

    def graph_replays(self):
        n = c_u64()
        check(load().fheon_server_graph_replays(self.handle.h, ctypes.byref(n)))
        return n.value

    def stats(self):
        st, mb, a, w = c_u64(), c_u32(), c_u32(), c_u32()
        check(load().fheon_server_stats(self.handle.h, ctypes.byref(st), ctypes.byref(mb), ctypes.byref(a),
                                        ctypes.byref(w)))
        return {"steps": st.value, "max_batch": mb.value, "active": a.value, "waiting": w.value}

    def model_stats(self, model):
        mb, mw, held = c_u32(), c_u64(), c_sz()
        check(load().fheon_server_model_stats(self.handle.h, model.h, ctypes.byref(mb), ctypes.byref(mw),
                                              ctypes.byref(held)))
        return {"max_batch": mb.value, "mem_waits": mw.value, "held": held.value}

    def close(self):
        self.handle.close()


class Handle:
    """Owning pointer to a fheon_* object, destroyed with its C destructor."""

    def __init__(self, h, destroy):
        self.h = h
        self._destroy = destroy

    def close(self):
        if self.h is not None and self.h.value:
            self._destroy(self.h)
        self.h = None

    def __del__(self):
        if sys is None or sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass
