"""Build and load the plain-C oracle (ckks_oracle.c) through ctypes.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libckks_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile ckks_oracle.c with gcc (plain -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
u32p = ctypes.POINTER(ctypes.c_uint32)
dblp = ctypes.POINTER(ctypes.c_double)
vp = ctypes.c_void_p
U32, U64, I32, DBL = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double

_SIGS = {
    "oracle_is_prime": (I32, [U64]),
    "oracle_gen_primes": (I32, [U32, u32p, U32, u64p]),
    "oracle_min_psi": (U64, [U64, U32]),
    "oracle_chacha20_block": (None, [u32p, U32, u32p, u32p]),
    "oracle_draw64": (U64, [U64, U32, U64, U64]),
    "oracle_cdt_table": (None, [DBL, I32, u64p]),
    "oracle_sample_ternary": (None, [U64, U32, U64, U32, i64p]),
    "oracle_sample_gauss": (None, [U64, U32, U64, U32, i64p]),
    "oracle_sample_uniform": (None, [U64, U32, U64, U32, U64, u64p]),
    "oracle_ntt_def": (None, [u64p, U32, U64, U64, u64p]),
    "oracle_intt_def": (None, [u64p, U32, U64, U64, u64p]),
    "oracle_ntt": (None, [u64p, U32, U64, U64, u64p]),
    "oracle_intt": (None, [u64p, U32, U64, U64, u64p]),
    "oracle_negacyclic_mul": (None, [u64p, u64p, U32, U64, u64p]),
    "oracle_automorph_coeff": (None, [u64p, U32, U64, U64, u64p]),
    "oracle_bconv": (None, [u64p, u64p, U32, u64p, U32, U32, u64p]),
    "oracle_ctx_new": (vp, [U32, u64p, U32, u64p, U32, U32, U64]),
    "oracle_ctx_free": (None, [vp]),
    "oracle_ctx_alpha": (U32, [vp]),
    "oracle_ctx_beta": (U32, [vp]),
    "oracle_ctx_psi": (U64, [vp, U32]),
    "oracle_keygen_sk": (None, [vp, i64p, u64p]),
    "oracle_keygen_pk": (None, [vp, u64p, u64p]),
    "oracle_keygen_ksk": (None, [vp, u64p, u64p, U64, u64p]),
    "oracle_galois_sk": (None, [vp, u64p, U64, u64p]),
    "oracle_to_coeff": (None, [vp, u64p, U32, I32, u64p]),
    "oracle_to_eval": (None, [vp, u64p, U32, I32, u64p]),
    "oracle_automorph_eval": (None, [vp, u64p, U32, I32, U64, u64p]),
    "oracle_modup": (None, [vp, u64p, U32, U32, u64p]),
    "oracle_moddown": (None, [vp, u64p, U32, u64p]),
    "oracle_keyswitch": (None, [vp, u64p, U32, u64p, u64p]),
    "oracle_rotate": (None, [vp, u64p, U32, U64, u64p, u64p]),
    "oracle_rotate_hoisted": (None, [vp, u64p, U32, u64p, U32, u64p, u64p]),
    "oracle_mul_relin": (None, [vp, u64p, u64p, U32, u64p, u64p]),
    "oracle_mul_int": (None, [vp, u64p, U32, ctypes.c_int64, u64p]),
    "oracle_add_int": (None, [vp, u64p, U32, ctypes.c_int64, u64p]),
    "oracle_const_factor": (ctypes.c_int64, [vp, U32, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "oracle_llround": (ctypes.c_int64, [ctypes.c_double]),
    "oracle_cheb_coeffs": (None, [ctypes.c_double, U32, ctypes.POINTER(ctypes.c_double)]),
    "oracle_cos_cheb_coeffs": (None, [ctypes.c_double, U32, U32, ctypes.POINTER(ctypes.c_double)]),
    "oracle_encrypt": (None, [vp, u64p, i64p, U64, u64p]),
    "oracle_plain_from_coeffs": (None, [vp, i64p, U32, u64p]),
    "oracle_decrypt": (None, [vp, u64p, u64p, U32, u64p]),
    "oracle_mul_plain": (None, [vp, u64p, u64p, U32, u64p]),
    "oracle_add": (None, [vp, u64p, u64p, U32, u64p]),
    "oracle_add_plain": (None, [vp, u64p, u64p, U32, u64p]),
    "oracle_rescale_poly": (None, [vp, u64p, U32, u64p]),
    "oracle_rescale": (None, [vp, u64p, U32, u64p]),
    "oracle_encode": (I32, [U32, dblp, dblp, U32, DBL, i64p]),
    "oracle_decode": (None, [U32, dblp, U32, DBL, dblp, dblp]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib
