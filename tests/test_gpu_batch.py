"""Batched statistics over many columns, and the dnum autotuner (N = 2^12).

The batched workload's shape at a size the oracle-backed checks finish
quickly: columns of uneven lengths, in pairs of a lognormal-shaped column
correlated with a Bernoulli column, all
five statistics per column (Pearson per pair) run as one batch; every result
equals the same query run alone, limb for limb, and decrypts within 1e-3 of
FP64.
"""
import json

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

DEEP12 = dict(log_n=12, n_q=20, n_p=2, dnum=10, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)


def columns(ctx, evk, count, seed):
    lens = workloads.log_uniform_lengths(count // 2, 100, 2048, seed=seed)
    cols, data = [], []
    for i in range(0, count, 2):
        b, y = workloads.pcc_pair(int(lens[i // 2]), seed=seed + i)  # y: lognormal-shaped, b: Bernoulli
        for j, x in enumerate((y, b)):
            cols.append(ctx.encrypt_column(evk, x, seed + 50 + i + j))
            data.append(x)
    return cols, data


def test_batched_columns_all_statistics():
    import paper_2508_12093_gb300 as pp
    from oracle import stats as ost
    ctx = pp.Context(DEEP12)
    sk, evk = ctx.keygen(4)
    cols, data = columns(ctx, evk, 8, 900)
    qs = []
    for i, c in enumerate(cols):
        B = 20.0 if i % 2 == 0 else 1.0
        for st in ("zscore", "cv", "skew", "kurt"):
            qs.append((st, c, None, dict(B_x=B, cheb_log2deg=5, newton_steps=2), (i,)))
    for i in range(0, len(cols), 2):
        qs.append(("pcc", cols[i], cols[i + 1], dict(B_x=20.0, B_y=1.0, cheb_log2deg=5, newton_steps=2), (i, i + 1)))
    batch = ctx.query_batch(evk, [q[:4] for q in qs])
    for q, rb in zip(qs, batch):
        rs = ctx.query(evk, *q[:4])
        for a, b in zip(rb.cts(), rs.cts()):
            a, b = ctx.ct_export(a), ctx.ct_export(b)
            assert a[2:] == b[2:] and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), q[0]
        vals, _ = ctx.decrypt(sk, rb)
        if q[0] == "pcc":
            want = np.array([ost.plain_stats(data[q[4][0]], data[q[4][1]])["pcc"]])
        else:
            ref = ost.plain_stats(data[q[4][0]])
            want = ref["znorm"] if q[0] == "zscore" else np.array([ref[q[0]]])
        assert np.abs(vals[:len(want)] - want).max() / np.abs(want).max() < 1e-3, (q[0], q[4])


def test_autotune_picks_a_measured_dnum(tmp_path):
    from paper_2508_12093_gb300 import autotune
    base = dict(log_n=12, n_q=12, n_p=2, dnum=6, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
    cache = str(tmp_path / "tuned.json")
    q = ("cv", dict(B_x=20.0, cheb_log2deg=3, newton_steps=1))  # depth 9 of the 11 levels
    best, table = autotune.tune(base, cache=cache, candidates=(2, 3, 6), reps=3, query=q)
    assert best in (2, 3, 6) and [r["dnum"] for r in table] == [2, 3, 6]
    for r in table:
        assert r["hmult_us"] > 0 and r["rotate_us"] > 0 and r["query_us"] > 0
        assert r["tile"] in (4, 8, 16) and r["hmult_us"] == min(r["tile_us"].values())
    fastest = min(table, key=lambda r: r["query_us"])["dnum"]
    assert best == fastest
    with open(cache) as f:
        assert list(json.load(f).values())[0]["dnum"] == best
    again, _ = autotune.tune(base, cache=cache, candidates=(2, 3, 6), reps=3, query=q)  # from the cache
    assert again == best
    assert autotune.tuned_params(base, cache=cache)["n_p"] == 12 // best
    prm, row = autotune.tuned_setup(base, cache=cache)
    assert prm["dnum"] == best and row["tile"] == next(r["tile"] for r in table if r["dnum"] == best)
    assert row["pass_min_blocks"] in autotune.PASS_BLOCKS and row["inner"]["words"] == 16  # N = 2^12


def test_many_queries_deterministic_full_size():
    """96 mixed queries of the 64-column workload at N = 2^16 with digits of 8
    primes (dnum = 3), run one at a time and through the request loop (32 in
    flight): every result identical in both forms and within 1e-3 of FP64. Guards
    against ordering races between consecutive launches."""
    import bench
    import paper_2508_12093_gb300 as pp
    from oracle import stats as ost
    from paper_2508_12093_gb300 import autotune
    ctx = pp.Context(autotune.with_dnum(workloads.PARAMS["n16_d6"], 3))
    sk, evk = ctx.keygen(2)
    cols, data = bench.batched_columns(ctx, evk)
    qs = bench.batched_queries(cols)[:96]
    serial = [ctx.query(evk, *q[:4]) for q in qs]
    srv = pp.Server(ctx, evk, 48 << 30, 32)
    ts = [srv.submit(*q[:4]) for q in qs]
    served = [srv.wait(t) for t in ts]
    srv.close()
    for q, a, b in zip(qs, serial, served):
        for x, y in zip(a.cts(), b.cts()):
            x, y = ctx.ct_export(x), ctx.ct_export(y)
            assert x[2:] == y[2:] and np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]), (q[0], q[4])
        vals, _ = ctx.decrypt(sk, b)
        if q[0] == "pcc":
            want = np.array([ost.plain_stats(data[q[4][0]], data[q[4][1]])["pcc"]])
        else:
            ref = ost.plain_stats(data[q[4][0]])
            want = ref["znorm"] if q[0] == "zscore" else np.array([ref[q[0]]])
        assert np.abs(vals[:len(want)] - want).max() / np.abs(want).max() < 1e-3, (q[0], q[4])
