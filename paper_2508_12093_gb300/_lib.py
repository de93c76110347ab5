"""ctypes binding of libppst.so (include/ppst.h): argument marshalling only.

Every function of the C ABI is exposed under its own name on `lib`. The
library must have been built (paper_2508_12093_gb300.build.build(), or
__graft_entry__.build()); importing without it raises ImportError -- there is
no CPU fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libppst.so")

c_void_p, c_int, c_size_t, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
c_u32, c_u64, c_i32, c_i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
P = ctypes.POINTER
PP = P(c_void_p)

PPST_OK = 0
ERRORS = {-1: "PPST_E_ARG", -2: "PPST_E_DEPTH", -3: "PPST_E_SCALE", -4: "PPST_E_OOM", -5: "PPST_E_BUDGET",
          -6: "PPST_E_CUDA", -7: "PPST_E_TIMEOUT", -8: "PPST_E_STATE"}
PPST_ZSCORE, PPST_CV, PPST_SKEW, PPST_KURT, PPST_PCC, PPST_CV_SIGNED = 0, 1, 2, 3, 4, 5


class ppst_params(ctypes.Structure):
    _fields_ = [("log_n", c_u32), ("n_q", c_u32), ("n_p", c_u32), ("dnum", c_u32), ("q0_bits", c_u32),
                ("q_bits", c_u32), ("p_bits", c_u32), ("log_scale", c_double), ("sigma", c_double),
                ("gauss_bound", c_u32)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_void_p, c_size_t, c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_size_t, c_void_p)


class ppst_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("user", c_void_p)]


class ppst_qopts(ctypes.Structure):
    _fields_ = [("B_x", c_double), ("B_y", c_double), ("cheb_log2deg", c_i32), ("newton_steps", c_i32)]


class ppst_report(ctypes.Structure):
    _fields_ = [("level_in", c_i32), ("level_out", c_i32), ("depth_used", c_i32), ("scale", c_double),
                ("n_cts", c_u32)]


class ppst_server_stats(ctypes.Structure):
    _fields_ = [("budget", c_size_t), ("reserved", c_size_t), ("held", c_size_t), ("running", c_u32),
                ("queued", c_u32)]


u64p, i64p, f64p, i32p, u32p = P(c_u64), P(c_i64), P(ctypes.c_double), P(c_i32), P(c_u32)

SIGNATURES = {
    "ppst_ctx_create": (c_int, [P(ppst_params), P(ppst_allocator), c_void_p, PP]),
    "ppst_last_error": (ctypes.c_char_p, [c_void_p]),
    "ppst_ctx_primes": (c_int, [c_void_p, u64p, c_size_t, u32p]),
    "ppst_sync": (c_int, [c_void_p]),
    "ppst_mem_info": (c_int, [c_void_p, P(c_size_t), P(c_size_t)]),
    "ppst_keygen": (c_int, [c_void_p, c_u64, i32p, c_size_t, PP, PP]),
    "ppst_sk_export": (c_int, [c_void_p, c_void_p, i64p, c_size_t]),
    "ppst_evk_export": (c_int, [c_void_p, c_void_p, c_i32, c_u32, u64p, u64p]),
    "ppst_encrypt_column": (c_int, [c_void_p, c_void_p, f64p, c_size_t, c_u64, PP]),
    "ppst_encrypt_ints": (c_int, [c_void_p, c_void_p, i64p, c_u64, c_u32, c_double, PP]),
    "ppst_decrypt": (c_int, [c_void_p, c_void_p, c_void_p, f64p, c_size_t, P(c_size_t), P(ppst_report)]),
    "ppst_decrypt_ct": (c_int, [c_void_p, c_void_p, c_void_p, f64p, c_size_t]),
    "ppst_query": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, P(ppst_qopts), PP]),
    "ppst_query_batch": (c_int, [c_void_p, c_void_p, c_size_t, P(c_int), PP, PP, P(ppst_qopts), PP]),
    "ppst_res_count": (c_int, [c_void_p, u32p]),
    "ppst_res_ct": (c_int, [c_void_p, c_u32, PP]),
    "ppst_col_from_cts": (c_int, [c_void_p, PP, c_size_t, c_size_t, PP]),
    "ppst_col_info": (c_int, [c_void_p, P(c_size_t), u32p]),
    "ppst_col_ct": (c_int, [c_void_p, c_u32, PP]),
    "ppst_ct_import": (c_int, [c_void_p, u64p, u64p, c_u32, c_double, PP]),
    "ppst_ct_export": (c_int, [c_void_p, c_void_p, u64p, u64p, u32p, f64p]),
    "ppst_ct_level": (c_int, [c_void_p, u32p, f64p]),
    "ppst_hmult": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, PP]),
    "ppst_hmult_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ppst_rotate": (c_int, [c_void_p, c_void_p, c_void_p, c_i32, PP]),
    "ppst_hmult_batch": (c_int, [c_void_p, c_void_p, c_size_t, PP, PP, PP]),
    "ppst_rotate_batch": (c_int, [c_void_p, c_void_p, c_size_t, PP, c_i32, PP]),
    "ppst_rotsum": (c_int, [c_void_p, c_void_p, c_void_p, PP]),
    "ppst_selftest_wait": (c_int, [c_void_p, c_u32]),
    "ppst_ctx_set_tile": (c_int, [c_void_p, c_u32]),
    "ppst_ctx_set_pass_blocks": (c_int, [c_void_p, c_u32]),
    "ppst_ctx_set_inner_shape": (c_int, [c_void_p, c_u32, c_u32]),
    "ppst_inv_sqrt": (c_int, [c_void_p, c_void_p, c_void_p, c_double, ctypes.c_int32, ctypes.c_int32, PP]),
    "ppst_rescale": (c_int, [c_void_p, c_void_p, PP]),
    "ppst_add": (c_int, [c_void_p, c_void_p, c_void_p, PP]),
    "ppst_sub": (c_int, [c_void_p, c_void_p, c_void_p, PP]),
    "ppst_add_const": (c_int, [c_void_p, c_void_p, c_double, PP]),
    "ppst_mul_const": (c_int, [c_void_p, c_void_p, c_double, c_double, PP]),
    "ppst_mul_int": (c_int, [c_void_p, c_void_p, c_i64, PP]),
    "ppst_drop": (c_int, [c_void_p, c_void_p, c_u32, PP]),
    "ppst_lin_comb": (c_int, [c_void_p, PP, f64p, c_size_t, c_double, PP]),
    "ppst_server_create": (c_int, [c_void_p, c_void_p, c_size_t, c_u32, PP]),
    "ppst_submit": (c_int, [c_void_p, c_int, c_void_p, c_void_p, P(ppst_qopts), P(c_u64)]),
    "ppst_wait": (c_int, [c_void_p, c_u64, c_i32, PP]),
    "ppst_ticket_latency": (c_int, [c_void_p, c_u64, P(c_double)]),
    "ppst_server_info": (c_int, [c_void_p, P(ppst_server_stats)]),
    "ppst_server_estimate": (c_int, [c_void_p, c_int, c_void_p, c_void_p, P(c_size_t), P(c_size_t)]),
    "ppst_query_prepare": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, P(ppst_qopts), PP]),
    "ppst_plan_run": (c_int, [c_void_p, PP]),
    "ppst_prof_start": (c_int, [c_void_p, ctypes.c_char_p]),
    "ppst_prof_stop": (c_int, [c_void_p]),
    "ppst_prof_read": (c_int, [c_void_p, ctypes.c_char_p, P(c_u64), P(ctypes.c_double), P(c_u64), P(c_u64)]),
    "ppst_launch_count": (c_int, [c_void_p, P(c_u64)]),
    "ppst_prof_classes": (c_int, [c_void_p, ctypes.c_char_p, c_size_t]),
    "ppst_free": (None, [c_void_p]),
}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libppst.so not built ({path}); run paper_2508_12093_gb300.build.build() "
                          "(the GPU path has no CPU fallback)")
    so = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(so, name)
        fn.restype = res
        fn.argtypes = args
    return so


lib = load()
