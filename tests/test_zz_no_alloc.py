"""ppst_hmult_noalloc, the HMult for callers that cannot allocate device memory
while running (a host whose allocator already owns the free HBM, a serving
thread that cannot absorb cudaMalloc's synchronisation).

Called through the C ABI and compared with ppst_hmult limb for limb (the
tolerance of every GPU parity test here: bit-exact) on two calls in a row, the
second with other operands at another level, so stale contents of the shared
static scratch array cannot leak into a result. This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

PRM = dict(log_n=12, n_q=20, n_p=2, dnum=10, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)


def export(ctx, ct):
    return ctx.ct_export(ct)


def test_noalloc_hmult_equals_hmult_twice():
    import paper_2508_12093_gb300 as pp
    from paper_2508_12093_gb300._lib import lib

    ctx = pp.Context(PRM)
    sk, evk = ctx.keygen(5, rotations=[1])
    x = workloads.uniform_column(ctx.S, seed=1, lo=-1.0, hi=1.0)
    y = workloads.uniform_column(ctx.S, seed=2, lo=-1.0, hi=1.0)
    a = ctx.encrypt_column(evk, x, 11).cts()[0]
    b = ctx.encrypt_column(evk, y, 12).cts()[0]
    # a ciphertext the caller already owns; its contents get replaced
    out = ctx.encrypt_ints(evk, np.zeros(ctx.N, dtype=np.int64), 13, 0, 2.0 ** 40)
    cases = [(a, b), (ctx.drop(b, 7), ctx.drop(a, 9))]
    # a first call loads the kernels it launches (CUDA loads kernels lazily)
    assert lib.ppst_hmult_noalloc(ctx.ptr, evk.ptr, a.ptr, b.ptr, out.ptr) == 0
    ctx.sync()
    for ca, cb in cases:
        in_use0, cached0 = ctx.mem_info()
        free0 = torch.cuda.mem_get_info()[0]
        rc = lib.ppst_hmult_noalloc(ctx.ptr, evk.ptr, ca.ptr, cb.ptr, out.ptr)
        assert rc == 0, lib.ppst_last_error(ctx.ptr)
        ctx.sync()
        assert ctx.mem_info() == (in_use0, cached0), "the pool was touched"
        assert torch.cuda.mem_get_info()[0] == free0, "device memory was allocated"
        want = ctx.hmult(evk, ca, cb)
        g0, g1, glv, gsc = export(ctx, out)
        w0, w1, wlv, wsc = export(ctx, want)
        assert (glv, gsc) == (wlv, wsc)
        assert np.array_equal(g0, w0) and np.array_equal(g1, w1)
        assert np.abs(ctx.decrypt_ct(sk, out) - x * y).max() < 1e-5


def test_noalloc_rejects_oversized_parameters_and_aliasing():
    import paper_2508_12093_gb300 as pp
    from paper_2508_12093_gb300._lib import lib

    big = pp.Context(workloads.PARAMS["n16_d6"])
    sk, evk = big.keygen(2, rotations=[1])
    a = big.encrypt_column(evk, workloads.uniform_column(100, seed=3), 1).cts()[0]
    out = big.encrypt_ints(evk, np.zeros(big.N, dtype=np.int64), 2, 0, 2.0 ** 50)
    assert lib.ppst_hmult_noalloc(big.ptr, evk.ptr, a.ptr, a.ptr, out.ptr) == -1
    assert b"MiB of scratch" in lib.ppst_last_error(big.ptr)
    small = pp.Context(PRM)
    sk2, evk2 = small.keygen(5, rotations=[1])
    c = small.encrypt_column(evk2, workloads.uniform_column(100, seed=4), 1).cts()[0]
    d = small.encrypt_ints(evk2, np.zeros(small.N, dtype=np.int64), 2, 0, 2.0 ** 40)
    assert lib.ppst_hmult_noalloc(small.ptr, evk2.ptr, d.ptr, c.ptr, d.ptr) == -1   # out aliases an input
    # a call that fails leaves the output as it was
    before = small.ct_export(d)
    low = small.drop(c, 0)
    assert lib.ppst_hmult_noalloc(small.ptr, evk2.ptr, low.ptr, low.ptr, d.ptr) == -2
    after = small.ct_export(d)
    assert before[2:] == after[2:] and np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
