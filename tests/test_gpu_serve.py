"""Continuous-batching server through the C ABI (N = 2^12, depth 19).

Queries submitted at staggered times join the running schedule at op
boundaries; every result must equal, limb for limb, the same query run alone,
whatever it was batched with. Admission limits, timeouts and per-query errors
are exercised on the same context.
"""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

DEEP12 = dict(log_n=12, n_q=20, n_p=2, dnum=10, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
OPTS12 = dict(B_x=20.0, B_y=20.0, cheb_log2deg=5, newton_steps=2)
GB = 1 << 30


@pytest.fixture(scope="module")
def env():
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(DEEP12)
    sk, evk = ctx.keygen(3)
    x = workloads.lognormal_column(1500, seed=11)
    x2, y2 = workloads.pcc_pair(2048, seed=12)
    cols = dict(x=ctx.encrypt_column(evk, x, 51), long=ctx.encrypt_column(evk, workloads.lognormal_column(6000, 13), 52),
                px=ctx.encrypt_column(evk, x2, 53), py=ctx.encrypt_column(evk, y2, 54))
    return pp, ctx, sk, evk, cols


def same(ctx, ra, rb):
    ga, gb = ra.cts(), rb.cts()
    assert len(ga) == len(gb)
    for a, b in zip(ga, gb):
        a, b = ctx.ct_export(a), ctx.ct_export(b)
        assert a[2:] == b[2:] and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def mix(cols):
    pcc = dict(OPTS12, B_x=1.0)
    return [("kurt", cols["x"], None, OPTS12), ("skew", cols["long"], None, OPTS12),
            ("pcc", cols["px"], cols["py"], pcc), ("cv", cols["x"], None, OPTS12),
            ("zscore", cols["x"], None, OPTS12), ("kurt", cols["long"], None, OPTS12),
            ("cv", cols["long"], None, dict(OPTS12, cheb_log2deg=4, newton_steps=3))]


@pytest.mark.parametrize("max_batch", [16, 2])
def test_server_staggered_equals_alone(env, max_batch):
    pp, ctx, sk, evk, cols = env
    qs = mix(cols)
    srv = pp.Server(ctx, evk, hbm_budget=8 * GB, max_batch=max_batch)
    rng = np.random.default_rng(7)
    tickets = []
    for q in qs:
        tickets.append(srv.submit(*q))
        time.sleep(float(rng.uniform(0, 0.02)))  # arrivals land mid-schedule
    got = [srv.wait(t) for t in tickets]
    lat = [srv.latency(t) for t in tickets]
    srv.close()
    assert all(v > 0 for v in lat)
    for q, r in zip(qs, got):
        same(ctx, r, ctx.query(evk, *q))


def test_server_budget_admission(env):
    pp, ctx, sk, evk, cols = env
    # one single-ciphertext query fits the budget, two do not: they run one after another
    srv = pp.Server(ctx, evk, hbm_budget=100 << 20, max_batch=16)
    qs = [("kurt", cols["x"], None, OPTS12), ("cv", cols["x"], None, OPTS12), ("skew", cols["x"], None, OPTS12)]
    ts = [srv.submit(*q) for q in qs]
    rs = [srv.wait(t) for t in ts]
    for q, r in zip(qs, rs):
        same(ctx, r, ctx.query(evk, *q))
    srv.close()
    small = pp.Server(ctx, evk, hbm_budget=32 << 20, max_batch=16)
    with pytest.raises(pp.PpstError) as e:
        small.submit("kurt", cols["x"], None, OPTS12)  # over the budget on its own
    assert e.value.code == -5
    small.close()


def test_server_timeout_and_errors(env):
    pp, ctx, sk, evk, cols = env
    srv = pp.Server(ctx, evk, hbm_budget=8 * GB, max_batch=16)
    t = srv.submit("kurt", cols["long"], None, OPTS12)
    assert srv.wait(t, timeout_ms=0) is None  # a depth-19 program is not done within the submit call
    r = srv.wait(t)
    assert r is not None and srv.latency(t) > 0
    with pytest.raises(pp.PpstError) as e:
        srv.wait(t)  # handed over already
    assert e.value.code == -8
    with pytest.raises(pp.PpstError) as e:
        srv.wait(12345)
    assert e.value.code == -1
    with pytest.raises(pp.PpstError) as e:
        srv.submit("pcc", cols["x"], None, OPTS12)
    assert e.value.code == -1
    # a query that runs out of levels fails alone; its neighbour completes
    good = srv.submit("skew", cols["x"], None, OPTS12)
    try:
        bad = srv.submit("kurt", cols["x"], None, dict(OPTS12, cheb_log2deg=10))
        with pytest.raises(pp.PpstError) as e:
            srv.wait(bad)
        assert e.value.code == -2
    except pp.PpstError as err:
        assert err.code == -2
    same(ctx, srv.wait(good), ctx.query(evk, "skew", cols["x"], None, OPTS12))
    srv.close()


def test_server_close_with_work_in_flight(env):
    pp, ctx, sk, evk, cols = env
    srv = pp.Server(ctx, evk, hbm_budget=8 * GB, max_batch=4)
    for q in mix(cols):
        srv.submit(*q)
    srv.close()  # drains the queue, frees unclaimed results
    r = ctx.query(evk, "cv", cols["x"], None, OPTS12)  # the context stays usable
    assert len(r.cts()) == 1


def test_budget_counts_results_until_taken(env):
    """Admission counts a finished query's result ciphertexts until ppst_wait
    hands them over: with room for one query and its result only, the second
    query starts after the first result is taken, not when the first query
    finishes; every result still equals the query run alone."""
    pp, ctx, sk, evk, cols = env
    probe = pp.Server(ctx, evk, hbm_budget=8 * GB, max_batch=4)
    w, r = probe.estimate("kurt", cols["x"])
    assert w > 0 and r > 0
    wz, rz = probe.estimate("zscore", cols["long"])
    assert rz == 3 * r  # one result ciphertext per input ciphertext (6000 rows)
    probe.close()
    srv = pp.Server(ctx, evk, hbm_budget=w + r + r // 2, max_batch=4)
    t1 = srv.submit("kurt", cols["x"], None, OPTS12)
    t2 = srv.submit("cv", cols["x"], None, OPTS12)
    info = srv.info()
    assert info["budget"] == w + r + r // 2 and info["running"] == 1 and info["queued"] == 1
    deadline = time.time() + 60
    while srv.info()["held"] == 0 and time.time() < deadline:  # the first query finishes
        time.sleep(0.01)
    info = srv.info()
    assert info["held"] == r and info["running"] == 0 and info["queued"] == 1, info
    time.sleep(0.2)
    assert srv.info()["queued"] == 1  # still blocked: its result is not taken yet
    r1 = srv.wait(t1)
    r2 = srv.wait(t2)
    info = srv.info()
    assert info["held"] == 0 and info["reserved"] == 0 and info["running"] == 0 and info["queued"] == 0
    same(ctx, r1, ctx.query(evk, "kurt", cols["x"], None, OPTS12))
    same(ctx, r2, ctx.query(evk, "cv", cols["x"], None, OPTS12))
    srv.close()


def test_small_query_passes_a_blocked_large_one_for_a_while(env):
    """A query that does not fit next to the running one is passed by a smaller
    one that does, and all three complete, each equal to the query alone."""
    pp, ctx, sk, evk, cols = env
    probe = pp.Server(ctx, evk, hbm_budget=8 * GB, max_batch=4)
    wl, rl = probe.estimate("zscore", cols["long"])  # three ciphertexts: larger
    ws, rs = probe.estimate("cv", cols["x"])
    probe.close()
    assert wl > ws and rl == 3 * rs
    budget = 2 * ws + 3 * rs  # two small queries fit together; the large one fits only alone
    assert ws + wl + rl > budget >= wl + rl and 2 * (ws + rs) <= budget
    srv = pp.Server(ctx, evk, hbm_budget=budget, max_batch=4)
    ta = srv.submit("cv", cols["x"], None, OPTS12)
    tb = srv.submit("zscore", cols["long"], None, OPTS12)  # blocked behind ta
    tc = srv.submit("kurt", cols["x"], None, OPTS12)       # fits beside ta: passes tb
    info = srv.info()
    assert info["running"] == 2 and info["queued"] == 1, info
    res = [srv.wait(t) for t in (ta, tb, tc)]
    for q, r in zip((("cv", cols["x"]), ("zscore", cols["long"]), ("kurt", cols["x"])), res):
        same(ctx, r, ctx.query(evk, q[0], q[1], None, OPTS12))
    srv.close()


def test_budget_from_free_device_memory(env):
    """hbm_budget = 0 takes the device's free memory (less a 5 % reserve)."""
    import torch
    pp, ctx, sk, evk, cols = env
    free, total = torch.cuda.mem_get_info()
    srv = pp.Server(ctx, evk, hbm_budget=0, max_batch=4)
    b = srv.info()["budget"]
    assert 0 < b <= free + ctx.mem_info()[1] and b >= free - total // 20 - (1 << 30)
    t = srv.submit("kurt", cols["x"], None, OPTS12)
    same(ctx, srv.wait(t), ctx.query(evk, "kurt", cols["x"], None, OPTS12))
    srv.close()
