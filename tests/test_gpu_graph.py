"""Prepared queries: the statistic program captured once as a CUDA graph and
replayed. Every replay's result equals ppst_query's for the same inputs, limb
for limb (N = 2^12, depth 19), across statistics, multi-ciphertext columns and
repeated replays; the context stays usable for ordinary calls in between."""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

DEEP12 = dict(log_n=12, n_q=20, n_p=2, dnum=10, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
OPTS12 = dict(B_x=20.0, B_y=20.0, cheb_log2deg=5, newton_steps=2)


@pytest.fixture(scope="module")
def env():
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(DEEP12)
    sk, evk = ctx.keygen(6)
    x = workloads.lognormal_column(1800, seed=21)
    long = workloads.lognormal_column(5000, seed=22)
    bx, by = workloads.pcc_pair(3000, seed=23)
    cols = dict(x=ctx.encrypt_column(evk, x, 61), long=ctx.encrypt_column(evk, long, 62),
                bx=ctx.encrypt_column(evk, bx, 63), by=ctx.encrypt_column(evk, by, 64))
    return pp, ctx, sk, evk, cols


def same(ctx, ra, rb):
    ga, gb = ra.cts(), rb.cts()
    assert len(ga) == len(gb)
    for a, b in zip(ga, gb):
        a, b = ctx.ct_export(a), ctx.ct_export(b)
        assert a[2:] == b[2:] and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("q", [("kurt", "x", None, OPTS12), ("zscore", "long", None, OPTS12),
                               ("cv", "long", None, OPTS12), ("pcc", "by", "bx", dict(OPTS12, B_y=1.0))])
def test_plan_replays_equal_query(env, q):
    pp, ctx, sk, evk, cols = env
    x, y = cols[q[1]], (cols[q[2]] if q[2] else None)
    want = ctx.query(evk, q[0], x, y, q[3])
    plan = ctx.prepare(evk, q[0], x, y, q[3])
    r1 = plan.run()
    r2 = plan.run()
    same(ctx, r1, want)
    same(ctx, r2, want)
    other = ctx.query(evk, "skew", cols["x"], None, OPTS12)  # ordinary calls in between
    r3 = plan.run()
    same(ctx, r3, want)
    same(ctx, other, ctx.query(evk, "skew", cols["x"], None, OPTS12))
    del r1
    plan.close()
    same(ctx, r2, want)  # results outlive the plan


def test_plan_is_faster_and_errors(env):
    pp, ctx, sk, evk, cols = env
    plan = ctx.prepare(evk, "kurt", cols["x"], None, OPTS12)
    for _ in range(3):
        plan.run(), ctx.query(evk, "kurt", cols["x"], None, OPTS12)
    ctx.sync()
    t0 = time.perf_counter()
    for _ in range(10):
        ctx.query(evk, "kurt", cols["x"], None, OPTS12)
    ctx.sync()
    t1 = time.perf_counter()
    for _ in range(10):
        plan.run()
    ctx.sync()
    t2 = time.perf_counter()
    print(f"kurtosis at N=2^12: query {1e3 * (t1 - t0) / 10:.2f} ms, graph replay {1e3 * (t2 - t1) / 10:.2f} ms")
    assert (t2 - t1) < (t1 - t0)
    with pytest.raises(pp.PpstError) as e:
        ctx.prepare(evk, "kurt", cols["x"], None, dict(OPTS12, cheb_log2deg=10))  # out of levels
    assert e.value.code == -2
    ctx.query(evk, "cv", cols["x"], None, OPTS12)  # the failed capture left the context usable
