"""One whole kurtosis query at N = 2^16 against the oracle, limb for limb.

The benchmark's settings (dnum = 6, B = 20, degree 127, 3 Newton steps, depth
19) on a 32,768-row lognormal column. The oracle's side (about ten minutes of
CPU time: fifteen Galois keys and the whole schedule) runs in a spawned worker
started at collection (tests/oracle_jobs.py); this file is collected after
the other GPU tests so that the job runs while they do.
"""
import pytest

import oracle_jobs as oj
import workloads

pytestmark = pytest.mark.gpu


def oj_check(ctx, g, want, what):
    from test_gpu_parity16 import check
    check(ctx, g, want, what)


def oj_imp(ctx, raw):
    c0, c1, lv, sc = raw
    return ctx.ct_import(c0, c1, lv, sc)


@pytest.mark.slow
@pytest.mark.oracle16("kurt")
def test_kurtosis_query_full_size():
    import paper_2508_12093_gb300 as pp
    from oracle import stats as ost
    ctx = pp.Context(workloads.PARAMS["n16_d6"])
    sk, evk = ctx.keygen(2)
    want = oj.result("kurt")
    col = ctx.col_from_cts([oj_imp(ctx, r) for r in want["cts"]], want["n"])
    o = oj.KURT_OPTS
    res = ctx.query(evk, "kurt", col, opts=dict(B_x=o["B"], cheb_log2deg=o["k"], newton_steps=o["t"]))
    oj_check(ctx, res.cts()[0], want["res"], "kurtosis query")
    v, rep = ctx.decrypt(sk, res)
    x = workloads.lognormal_column(32768, seed=1)
    assert abs(v[0] / ost.plain_stats(x)["kurt"] - 1) < 1e-3
    assert rep["depth_used"] == 19
