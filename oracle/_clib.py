"""ctypes loader for the oracle's C primitives (oracle/ckks_oracle.c).

TEST INFRASTRUCTURE. Only tests, the smoke check and the benchmark's CPU
baseline may import the oracle. `build()` compiles the C file with gcc into
oracle/_build/; loading fails loudly if that has not happened.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libppst_oracle.so")


def build(force=False):
    """Compile the oracle's C primitives (plain gcc, no GPU, no CUDA)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    # -ffp-contract=off: the Gaussian table is evaluated in plain IEEE double
    # without fused multiply-add, in the order the source states.
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", _SO, _SRC, "-lm"]
    subprocess.check_call(cmd)
    return _SO


u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
u32p = ctypes.POINTER(ctypes.c_uint32)
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def _load():
    if not os.path.exists(_SO):
        build()
    lib = ctypes.CDLL(_SO)
    sig = {
        "or_powmod": (_u64, [_u64, _u64, _u64]),
        "or_invmod": (_u64, [_u64, _u64]),
        "or_is_prime": (ctypes.c_int, [_u64]),
        "or_ntt_fwd": (None, [u64p, _u32, _u64, _u64]),
        "or_ntt_inv": (None, [u64p, _u32, _u64, _u64]),
        "or_ntt_fwd_batch": (None, [u64p, _u32, _u32, u64p, u64p]),
        "or_ntt_inv_batch": (None, [u64p, _u32, _u32, u64p, u64p]),
        "or_vec_mul": (None, [u64p, u64p, u64p, _u32, _u32, u64p]),
        "or_vec_mul_scalar": (None, [u64p, u64p, u64p, _u32, _u32, u64p]),
        "or_poly_mul": (None, [u64p, u64p, u64p, _u32, _u32, u64p, u64p]),
        "or_automorph": (None, [u64p, u64p, _u32, _u32, u64p, _u64]),
        "or_bconv": (None, [u64p, u64p, _u32, u64p, u64p, _u32, _u32]),
        "or_splitmix64": (_u64, [u64p]),
        "or_key_from_seed": (None, [_u64, u32p]),
        "or_chacha20_block": (None, [u32p, _u32, u32p, u32p]),
        "or_sample_uniform": (None, [_u64, _u32, _u32, _u32, _u64, _u32, u64p]),
        "or_sample_ternary": (None, [_u64, _u32, _u32, _u32, i64p]),
        "or_cdt_table": (None, [ctypes.c_double, _u32, u64p]),
        "or_sample_gauss": (None, [_u64, _u32, _u32, _u32, u64p, _u32, i64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def ptr64(a):
    """uint64 pointer to a C-contiguous numpy array (checked)."""
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(u64p)


def ptri64(a):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(i64p)


def ptr32(a):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(u32p)
