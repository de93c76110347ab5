"""GB300-native RNS-CKKS evaluator for PP-STAT's encrypted statistics.

A thin Python face of the C ABI in include/ppst.h (argument marshalling only:
every step runs in the CUDA library). PyTorch supplies device memory (through
its caching allocator) and the CUDA stream; numpy arrays carry host buffers.

    ctx = Context(workloads.PARAMS["n16_d6"])
    sk, evk = ctx.keygen(seed=2)
    col = ctx.encrypt_column(evk, x, seed=3)
    res = ctx.query(evk, PPST_KURT, col, opts=dict(B_x=20, cheb_log2deg=7, newton_steps=3))
    values, report = ctx.decrypt(sk, res)
"""
import ctypes
import weakref

import numpy as np

from . import _lib
from ._lib import (ERRORS, PPST_CV, PPST_CV_SIGNED, PPST_KURT, PPST_PCC, PPST_SKEW, PPST_ZSCORE, lib, ppst_allocator,  # noqa: F401
                   ppst_params, ppst_qopts, ppst_report)

STATS = {"zscore": PPST_ZSCORE, "cv": PPST_CV, "skew": PPST_SKEW, "kurt": PPST_KURT, "pcc": PPST_PCC,
         "cv_signed": PPST_CV_SIGNED}


class PpstError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(_lib.u64p)


class _Handle:
    def __init__(self, ctx, ptr):
        self.ctx, self.ptr = ctx, ptr
        live = getattr(ctx, "_live", None)
        if live is not None:
            live.add(self)  # closing the context frees the handle first

    def close(self):
        if self.ptr:
            lib.ppst_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SecretKey(_Handle):
    pass


class EvalKeys(_Handle):
    pass


class Ciphertext(_Handle):
    @property
    def level(self):
        lv, sc = _lib.c_u32(), ctypes.c_double()
        lib.ppst_ct_level(self.ptr, ctypes.byref(lv), ctypes.byref(sc))
        return lv.value

    @property
    def scale(self):
        lv, sc = _lib.c_u32(), ctypes.c_double()
        lib.ppst_ct_level(self.ptr, ctypes.byref(lv), ctypes.byref(sc))
        return sc.value


class Column(_Handle):
    def __init__(self, ctx, ptr, n):
        super().__init__(ctx, ptr)
        self.n = n

    def cts(self):
        n = _lib.c_u32()
        lib.ppst_col_info(self.ptr, None, ctypes.byref(n))
        out = []
        for i in range(n.value):
            p = ctypes.c_void_p()
            lib.ppst_col_ct(self.ptr, i, ctypes.byref(p))
            out.append(_View(self.ctx, p.value, self))
        return out


class Result(_Handle):
    def cts(self):
        n = _lib.c_u32()
        lib.ppst_res_count(self.ptr, ctypes.byref(n))
        out = []
        for i in range(n.value):
            p = ctypes.c_void_p()
            lib.ppst_res_ct(self.ptr, i, ctypes.byref(p))
            out.append(_View(self.ctx, p.value, self))
        return out


class _View(Ciphertext):
    """A ciphertext owned by a Result (not freed on its own)."""

    def __init__(self, ctx, ptr, owner):
        self.ctx, self.ptr, self._owner = ctx, ptr, owner

    def close(self):
        self.ptr = None


def _opts(o):
    if o is None:
        o = {}
    if isinstance(o, ppst_qopts):
        return o
    return ppst_qopts(float(o.get("B_x", 1.0)), float(o.get("B_y", 1.0)), int(o.get("cheb_log2deg", 7)),
                      int(o.get("newton_steps", 3)))


class Server(_Handle):
    """Continuous-batching request loop over one context and key set.

    Queries join the running schedule at the next evaluator-op boundary, so
    their HMults and rotate-and-sums share batched key-switch launches with
    the queries already in flight. Admission is bounded by an HBM budget and a
    maximum number of concurrent queries."""

    def __init__(self, ctx, evk, hbm_budget, max_batch=16):
        out = ctypes.c_void_p()
        ctx._check(lib.ppst_server_create(ctx.ptr, evk.ptr, int(hbm_budget), int(max_batch), ctypes.byref(out)))
        super().__init__(ctx, out.value)
        self.evk = evk
        self._rows = {}

    def submit(self, stat, x, y=None, opts=None):
        t = _lib.c_u64()
        o = _opts(opts)
        self.ctx._check(lib.ppst_submit(self.ptr, STATS.get(stat, stat), x.ptr, y.ptr if y is not None else None,
                                        ctypes.byref(o), ctypes.byref(t)))
        self._rows[t.value] = x.n if STATS.get(stat, stat) == PPST_ZSCORE else 1
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """The ticket's Result, or None on timeout (the ticket stays valid)."""
        out = ctypes.c_void_p()
        rc = lib.ppst_wait(self.ptr, ticket, int(timeout_ms), ctypes.byref(out))
        if rc == -7:  # PPST_E_TIMEOUT
            return None
        self.ctx._check(rc)
        r = Result(self.ctx, out.value)
        r.n = self._rows.pop(ticket)
        return r

    def latency(self, ticket):
        s = ctypes.c_double()
        self.ctx._check(lib.ppst_ticket_latency(self.ptr, ticket, ctypes.byref(s)))
        return s.value

    def info(self):
        """ppst_server_info as a dict: budget, reserved, held, running, queued."""
        o = _lib.ppst_server_stats()
        self.ctx._check(lib.ppst_server_info(self.ptr, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in o._fields_}

    def estimate(self, stat, x, y=None):
        """(working-set bytes, result bytes) that admission reserves for a query."""
        w, r = ctypes.c_size_t(), ctypes.c_size_t()
        self.ctx._check(lib.ppst_server_estimate(self.ptr, STATS.get(stat, stat), x.ptr,
                                                 y.ptr if y is not None else None, ctypes.byref(w), ctypes.byref(r)))
        return w.value, r.value


class Plan(_Handle):
    """A query captured as a CUDA graph (Context.prepare); run() replays it."""

    def __init__(self, ctx, ptr, rows):
        super().__init__(ctx, ptr)
        self.rows = rows

    def run(self):
        out = ctypes.c_void_p()
        self.ctx._check(lib.ppst_plan_run(self.ptr, ctypes.byref(out)))
        r = Result(self.ctx, out.value)
        r.n = self.rows
        return r


_CONTEXTS = weakref.WeakSet()
_ATEXIT = []


def _close_all():
    """Closes every open context before interpreter shutdown: a context returns
    its device memory through the torch allocator callbacks, which must run
    while torch is still alive."""
    for c in list(_CONTEXTS):
        try:
            c.close()
        except Exception:
            pass


class Context:
    """One parameter set on one GPU stream (not thread-safe)."""

    def __init__(self, params, use_torch=True, stream=None):
        self.params = dict(params)
        self._live = weakref.WeakSet()
        prm = ppst_params(params["log_n"], params["n_q"], params["n_p"], params["dnum"], params["q0_bits"],
                          params["q_bits"], params["p_bits"], float(params["log_scale"]),
                          float(params.get("sigma", 0.0)), int(params.get("gauss_bound", 0)))
        self._alloc = None
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("CUDA is not available: the library has no CPU path")
            dev = torch.cuda.current_device()
            self.stream = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)

            def _alloc(user, nbytes, strm):
                return torch.cuda.caching_allocator_alloc(nbytes, dev, strm or 0)

            def _release(user, ptr, nbytes, strm):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (_lib.ALLOC_FN(_alloc), _lib.RELEASE_FN(_release))
            self._alloc = ppst_allocator(self._cb[0], self._cb[1], None)
        else:
            self.stream = 0 if stream is None else int(stream)
        out = ctypes.c_void_p()
        rc = lib.ppst_ctx_create(ctypes.byref(prm), ctypes.byref(self._alloc) if self._alloc else None,
                                 ctypes.c_void_p(self.stream), ctypes.byref(out))
        if rc != 0:
            raise PpstError(rc, "ppst_ctx_create failed")
        self.ptr = out.value
        _CONTEXTS.add(self)
        if not _ATEXIT:  # registered after torch's own handlers, so it runs before them
            import atexit
            atexit.register(_close_all)
            _ATEXIT.append(True)
        n = _lib.c_u32()
        lib.ppst_ctx_primes(self.ptr, None, 0, ctypes.byref(n))
        buf = np.zeros(n.value, dtype=np.uint64)
        lib.ppst_ctx_primes(self.ptr, buf.ctypes.data_as(_lib.u64p), n.value, ctypes.byref(n))
        self.primes = [int(v) for v in buf]
        self.N = 1 << params["log_n"]
        self.S = self.N // 2
        self.L = params["n_q"] - 1
        self.K = params["n_p"]

    def close(self):
        """Frees every live handle of this context (servers first: they drain
        their queries), then the context itself."""
        if getattr(self, "ptr", None):
            live = list(getattr(self, "_live", ()))
            for h in live:
                if isinstance(h, (Server, Plan)):
                    h.close()
            for h in live:
                h.close()
            lib.ppst_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise PpstError(rc, lib.ppst_last_error(self.ptr).decode())

    def _new(self, fn, *args, cls=Ciphertext):
        out = ctypes.c_void_p()
        self._check(fn(self.ptr, *args, ctypes.byref(out)))
        return cls(self, out.value)

    # -- keys / encryption ----------------------------------------------------
    def keygen(self, seed, rotations=None):
        sk, evk = ctypes.c_void_p(), ctypes.c_void_p()
        if rotations:
            arr = (ctypes.c_int32 * len(rotations))(*rotations)
            rc = lib.ppst_keygen(self.ptr, seed, arr, len(rotations), ctypes.byref(sk), ctypes.byref(evk))
        else:
            rc = lib.ppst_keygen(self.ptr, seed, None, 0, ctypes.byref(sk), ctypes.byref(evk))
        self._check(rc)
        return SecretKey(self, sk.value), EvalKeys(self, evk.value)

    def sk_export(self, sk):
        s = np.zeros(self.N, dtype=np.int64)
        self._check(lib.ppst_sk_export(self.ptr, sk.ptr, s.ctypes.data_as(_lib.i64p), self.N))
        return s

    def evk_export(self, evk, which, digit):
        rows = self.L + 1 + self.K
        b = np.zeros((rows, self.N), dtype=np.uint64)
        a = np.zeros((rows, self.N), dtype=np.uint64)
        self._check(lib.ppst_evk_export(self.ptr, evk.ptr, which, digit, b.ctypes.data_as(_lib.u64p),
                                        a.ctypes.data_as(_lib.u64p)))
        return b, a

    def encrypt_column(self, evk, x, seed):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = ctypes.c_void_p()
        self._check(lib.ppst_encrypt_column(self.ptr, evk.ptr, x.ctypes.data_as(_lib.f64p), len(x), seed,
                                            ctypes.byref(out)))
        return Column(self, out.value, len(x))

    def encrypt_ints(self, evk, m, seed, index, scale):
        m = np.ascontiguousarray(m, dtype=np.int64)
        return self._new(lib.ppst_encrypt_ints, evk.ptr, m.ctypes.data_as(_lib.i64p), seed, index, float(scale))

    def decrypt(self, sk, res, cap=None):
        if cap is None:
            cap = max(1, getattr(res, "n", 1))
        out = np.zeros(cap, dtype=np.float64)
        n = ctypes.c_size_t()
        rep = ppst_report()
        self._check(lib.ppst_decrypt(self.ptr, sk.ptr, res.ptr, out.ctypes.data_as(_lib.f64p), cap,
                                     ctypes.byref(n), ctypes.byref(rep)))
        report = dict(level_in=rep.level_in, level_out=rep.level_out, depth_used=rep.depth_used,
                      scale=rep.scale, n_cts=rep.n_cts)
        return out[:min(cap, n.value)], report

    def decrypt_ct(self, sk, ct):
        out = np.zeros(self.S, dtype=np.float64)
        self._check(lib.ppst_decrypt_ct(self.ptr, sk.ptr, ct.ptr, out.ctypes.data_as(_lib.f64p), self.S))
        return out

    # -- statistics -----------------------------------------------------------
    def query(self, evk, stat, x, y=None, opts=None):
        stat = STATS.get(stat, stat)
        o = _opts(opts)
        out = ctypes.c_void_p()
        self._check(lib.ppst_query(self.ptr, evk.ptr, stat, x.ptr, y.ptr if y is not None else None,
                                   ctypes.byref(o), ctypes.byref(out)))
        r = Result(self, out.value)
        r.n = x.n if stat == PPST_ZSCORE else 1
        return r

    def prepare(self, evk, stat, x, y=None, opts=None):
        """The query captured as a CUDA graph: Plan.run() replays it."""
        o = _opts(opts)
        out = ctypes.c_void_p()
        st = STATS.get(stat, stat)
        self._check(lib.ppst_query_prepare(self.ptr, evk.ptr, st, x.ptr, y.ptr if y is not None else None,
                                           ctypes.byref(o), ctypes.byref(out)))
        return Plan(self, out.value, x.n if st == PPST_ZSCORE else 1)

    def query_batch(self, evk, queries):
        """queries: list of (stat, x, y_or_None, opts)."""
        n = len(queries)
        stats = (ctypes.c_int * n)(*[STATS.get(q[0], q[0]) for q in queries])
        xs = (ctypes.c_void_p * n)(*[q[1].ptr for q in queries])
        ys = (ctypes.c_void_p * n)(*[(q[2].ptr if q[2] is not None else None) for q in queries])
        opts = (ppst_qopts * n)(*[_opts(q[3]) for q in queries])
        outs = (ctypes.c_void_p * n)()
        self._check(lib.ppst_query_batch(self.ptr, evk.ptr, n, stats, xs, ys, opts, outs))
        res = []
        for q, p in zip(queries, outs):
            r = Result(self, p)
            r.n = q[1].n if STATS.get(q[0], q[0]) == PPST_ZSCORE else 1
            res.append(r)
        return res

    def col_from_cts(self, cts, n_rows):
        arr = (ctypes.c_void_p * len(cts))(*[c.ptr for c in cts])
        out = ctypes.c_void_p()
        self._check(lib.ppst_col_from_cts(self.ptr, arr, len(cts), n_rows, ctypes.byref(out)))
        return Column(self, out.value, n_rows)

    # -- ciphertext ops -------------------------------------------------------------
    def ct_import(self, c0, c1, level, scale):
        c0, p0 = _u64(c0)
        c1, p1 = _u64(c1)
        assert c0.shape == (level + 1, self.N) and c1.shape == c0.shape
        return self._new(lib.ppst_ct_import, p0, p1, level, float(scale))

    def ct_export(self, ct):
        lv, sc = _lib.c_u32(), ctypes.c_double()
        self._check(lib.ppst_ct_export(self.ptr, ct.ptr, None, None, ctypes.byref(lv), ctypes.byref(sc)))
        c0 = np.zeros((lv.value + 1, self.N), dtype=np.uint64)
        c1 = np.zeros_like(c0)
        self._check(lib.ppst_ct_export(self.ptr, ct.ptr, c0.ctypes.data_as(_lib.u64p), c1.ctypes.data_as(_lib.u64p),
                                       ctypes.byref(lv), ctypes.byref(sc)))
        return c0, c1, lv.value, sc.value

    def hmult(self, evk, a, b):
        return self._new(lib.ppst_hmult, evk.ptr, a.ptr, b.ptr)

    def hmult_noalloc(self, evk, a, b, out):
        """ppst_hmult_noalloc: writes a * b into the caller-owned ciphertext `out`."""
        self._check(lib.ppst_hmult_noalloc(self.ptr, evk.ptr, a.ptr, b.ptr, out.ptr))
        return out

    def rotate(self, evk, a, r):
        return self._new(lib.ppst_rotate, evk.ptr, a.ptr, r)

    def hmult_batch(self, evk, a_list, b_list):
        """ppst_hmult_batch: a_i * b_i for up to 16 pairs in one key-switch launch sequence."""
        n = len(a_list)
        pa = (ctypes.c_void_p * n)(*[x.ptr for x in a_list])
        pb = (ctypes.c_void_p * n)(*[x.ptr for x in b_list])
        out = (ctypes.c_void_p * n)()
        self._check(lib.ppst_hmult_batch(self.ptr, evk.ptr, n, pa, pb, out))
        return [Ciphertext(self, out[i]) for i in range(n)]

    def rotate_batch(self, evk, a_list, r):
        """ppst_rotate_batch: Rot(a_i, r) for up to 16 ciphertexts in one launch sequence."""
        n = len(a_list)
        pa = (ctypes.c_void_p * n)(*[x.ptr for x in a_list])
        out = (ctypes.c_void_p * n)()
        self._check(lib.ppst_rotate_batch(self.ptr, evk.ptr, n, pa, int(r), out))
        return [Ciphertext(self, out[i]) for i in range(n)]

    def rotsum(self, evk, a):
        return self._new(lib.ppst_rotsum, evk.ptr, a.ptr)

    def inv_sqrt(self, evk, v, C, cheb_log2deg=7, newton_steps=3):
        """CryptoInvSqrt: approximately 1/sqrt(C v) in every slot, v in (0, 2]."""
        return self._new(lib.ppst_inv_sqrt, evk.ptr, v.ptr, float(C), int(cheb_log2deg), int(newton_steps))

    def rescale(self, a):
        return self._new(lib.ppst_rescale, a.ptr)

    def add(self, a, b):
        return self._new(lib.ppst_add, a.ptr, b.ptr)

    def sub(self, a, b):
        return self._new(lib.ppst_sub, a.ptr, b.ptr)

    def add_const(self, a, x):
        return self._new(lib.ppst_add_const, a.ptr, float(x))

    def mul_const(self, a, x, target=0.0):
        return self._new(lib.ppst_mul_const, a.ptr, float(x), float(target or 0.0))

    def mul_int(self, a, k):
        return self._new(lib.ppst_mul_int, a.ptr, int(k))

    def lin_comb(self, cts, coeffs, target):
        arr = (ctypes.c_void_p * len(cts))(*[c.ptr for c in cts])
        cs = np.ascontiguousarray(coeffs, dtype=np.float64)
        return self._new(lib.ppst_lin_comb, arr, cs.ctypes.data_as(_lib.f64p), len(cts), float(target))

    def drop(self, a, level):
        return self._new(lib.ppst_drop, a.ptr, level)

    def set_tile(self, inner_sub):
        """Chunks per block of the key-switching inner product (4, 8 or 16)."""
        self._check(lib.ppst_ctx_set_tile(self.ptr, int(inner_sub)))
        self.inner_sub = int(inner_sub)


    def set_inner_shape(self, words_per_thread, lazy=False, shuffle=False, moddown8=False, modup8=False,
                        inverse8=False):
        """ppst_ctx_set_inner_shape: 16 or 8 words per thread in the inner product, lazy 128-bit
        accumulation and warp-shuffle exchanges (8 words only), 8-word ModDown CHUNKS pass, COLS
        passes and first inverse passes; speed only."""
        flags = (int(bool(lazy)) | (2 if shuffle else 0) | (4 if moddown8 else 0) | (8 if modup8 else 0)
                 | (16 if inverse8 else 0))
        self._check(lib.ppst_ctx_set_inner_shape(self.ptr, int(words_per_thread), flags))

    def set_pass_blocks(self, min_blocks):
        """ppst_ctx_set_pass_blocks: smaller transform blocks below this grid size (speed only)."""
        self._check(lib.ppst_ctx_set_pass_blocks(self.ptr, int(min_blocks)))
    def selftest_wait(self, timeout_us):
        """Launch a kernel whose bounded wait times out (failure-detection test);
        the next synchronising call raises PpstError(PPST_E_CUDA)."""
        self._check(lib.ppst_selftest_wait(self.ptr, int(timeout_us)))

    def sync(self):
        self._check(lib.ppst_sync(self.ptr))

    # -- kernel timing (CUDA events on the context's stream) ----------------------
    def prof_start(self, kernel_class=None):
        self._check(lib.ppst_prof_start(self.ptr, kernel_class.encode() if kernel_class else None))

    def prof_stop(self):
        self._check(lib.ppst_prof_stop(self.ptr))

    def prof_classes(self):
        buf = ctypes.create_string_buffer(4096)
        self._check(lib.ppst_prof_classes(self.ptr, buf, 4096))
        return [s for s in buf.value.decode().split(",") if s]

    def prof_read(self, kernel_class, with_units=False, with_method=False):
        """(launches, ms[, units][, method_units]) of a kernel class since prof_start."""
        n, ms, u, mu = _lib.c_u64(), ctypes.c_double(), _lib.c_u64(), _lib.c_u64()
        self._check(lib.ppst_prof_read(self.ptr, kernel_class.encode(), ctypes.byref(n), ctypes.byref(ms),
                                       ctypes.byref(u), ctypes.byref(mu)))
        out = (n.value, ms.value) + ((u.value,) if with_units else ()) + ((mu.value,) if with_method else ())
        return out

    def launch_count(self):
        n = _lib.c_u64()
        self._check(lib.ppst_launch_count(self.ptr, ctypes.byref(n)))
        return n.value

    def prof_read_all(self):
        return {k: self.prof_read(k) for k in self.prof_classes()}

    def mem_info(self):
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        lib.ppst_mem_info(self.ptr, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value
