"""GPU statistic queries through the C ABI.

* N = 2^12: every statistic's full schedule, result limbs bit-exact against
  the oracle, on one ciphertext and on a ragged two-ciphertext column;
* N = 2^16 (the 128-bit parameter set): decrypted statistics within 1e-3
  relative error of FP64 plaintext, and HMult + key switch bit-exact against
  the oracle at the top level.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

# N = 2^12, 20 Q primes (depth 19), 2 special primes, digits of 2 primes
DEEP12 = dict(log_n=12, n_q=20, n_p=2, dnum=10, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
OPTS12 = dict(B_x=20.0, B_y=20.0, cheb_log2deg=5, newton_steps=2)
TOL = 1e-3


@pytest.fixture(scope="module")
def deep():
    import paper_2508_12093_gb300 as pp
    from oracle import ckks as ock
    ctx = pp.Context(DEEP12)
    sk, evk = ctx.keygen(2)
    oc = ock.Ckks(ock.Params(**DEEP12))
    ok = oc.keygen(2, rotations=[1 << i for i in range(DEEP12["log_n"] - 1)])
    return ctx, sk, evk, oc, ok


def shared_column(env, x, seed):
    ctx, sk, evk, oc, ok = env
    o = oc.encrypt_column(ok["pk"], x, seed)
    g = [ctx.ct_import(c.c0, c.c1, c.level, c.scale) for c in o]
    return o, ctx.col_from_cts(g, len(x))


def check_same(ctx, g, o):
    c0, c1, lv, sc = ctx.ct_export(g)
    assert (lv, sc) == (o.level, o.scale)
    assert np.array_equal(c0, o.c0) and np.array_equal(c1, o.c1)


@pytest.mark.parametrize("n", [2048, 2048 + 301, 1, 2049])
@pytest.mark.parametrize("stat", ["skew", "kurt", "cv", "zscore"])
def test_schedule_parity_small(deep, stat, n):
    from oracle import stats as ost
    ctx, sk, evk, oc, ok = deep
    if n == 1 and stat != "cv":
        pytest.skip("a single row has zero variance")
    x = workloads.lognormal_column(n, seed=5)
    o, col = shared_column(deep, x, 21)
    res = ctx.query(evk, stat, col, opts=OPTS12)
    f = {"skew": ost.skew, "kurt": ost.kurt, "cv": ost.cv, "zscore": ost.znorm}[stat]
    if n == 1:
        return  # the variance is 0: outside the method's domain; the run itself must not fail
    want = f(ost.CkksEv(oc, ok), o, n, 20.0, 5, 2)
    want = want if isinstance(want, list) else [want]
    got = res.cts()
    assert len(got) == len(want)
    for g, w in zip(got, want):
        check_same(ctx, g, w)
    vals, rep = ctx.decrypt(sk, res)
    ref = ost.plain_stats(x)
    if stat == "zscore":
        assert len(vals) == n
        assert np.abs(vals - ref["znorm"]).max() / np.abs(ref["znorm"]).max() < TOL
    else:
        assert abs(vals[0] / ref[stat] - 1) < TOL
    assert rep["depth_used"] == DEEP12["n_q"] - 1 - rep["level_out"]


# the benchmark's approximation settings (degree 127, 3 Newton steps): depth 19 for
# skewness and kurtosis, the whole 20-prime chain
OPTS12_BENCH = dict(B_x=20.0, B_y=20.0, cheb_log2deg=7, newton_steps=3)


@pytest.mark.parametrize("stat", ["skew", "kurt", "cv", "zscore", "pcc"])
def test_schedule_parity_benchmark_settings(deep, stat):
    """Every statistic at degree 127 + 3 Newton steps (one Chebyshev split
    recursion deeper than degree 31) on a ragged two-ciphertext column: result
    limbs bit-exact against the oracle."""
    from oracle import stats as ost
    ctx, sk, evk, oc, ok = deep
    n = 2048 + 301
    o = OPTS12_BENCH
    if stat == "pcc":
        x, y = workloads.pcc_pair(n, seed=16)
        ox, cx = shared_column(deep, x, 61)
        oy, cy = shared_column(deep, y, 62)
        res = ctx.query(evk, "pcc", cx, cy, opts=dict(o, B_x=1.0))
        want = [ost.pcc(ost.CkksEv(oc, ok), ox, oy, n, 1.0, 20.0, o["cheb_log2deg"], o["newton_steps"])]
        ref = ost.plain_stats(x, y)["pcc"]
    else:
        x = workloads.lognormal_column(n, seed=15)
        ox, cx = shared_column(deep, x, 63)
        res = ctx.query(evk, stat, cx, opts=o)
        f = {"skew": ost.skew, "kurt": ost.kurt, "cv": ost.cv, "zscore": ost.znorm}[stat]
        want = f(ost.CkksEv(oc, ok), ox, n, 20.0, o["cheb_log2deg"], o["newton_steps"])
        want = want if isinstance(want, list) else [want]
        ref = ost.plain_stats(x)["znorm" if stat == "zscore" else stat]
    got = res.cts()
    assert len(got) == len(want)
    for g, w in zip(got, want):
        check_same(ctx, g, w)
    vals, rep = ctx.decrypt(sk, res)
    if stat == "zscore":
        assert np.abs(vals - ref).max() / np.abs(ref).max() < TOL
    else:
        assert abs(vals[0] / ref - 1) < TOL
    assert rep["depth_used"] == {"skew": 19, "kurt": 19, "cv": 17, "zscore": 17, "pcc": 18}[stat]


@pytest.mark.parametrize("mu,n,k,t", [(-3.0, 2048 + 301, 5, 2), (-3.0, 2048 + 301, 7, 3), (4.0, 2048, 7, 3),
                                       (-0.7, 2049, 5, 2)])
def test_sign_aware_cv_parity(deep, mu, n, k, t):
    """The sign-aware CV (Alg. 6 with Sign) on normal columns of either sign:
    result limbs bit-exact against the oracle, the value within 1e-3 of FP64
    (negative for a negative mean), one level more than the positive-mean CV
    (depth 18 at degree 127 + 3 Newton steps, in a 19-level chain)."""
    from oracle import stats as ost
    ctx, sk, evk, oc, ok = deep
    B = 6.0
    x = workloads.normal_column(n, seed=17, mu=mu, sigma=3.0)
    o, col = shared_column(deep, x, 71)
    opts = dict(B_x=B, cheb_log2deg=k, newton_steps=t)
    res = ctx.query(evk, "cv_signed", col, opts=opts)
    check_same(ctx, res.cts()[0], ost.cv_signed(ost.CkksEv(oc, ok), o, n, B, k, t))
    v, rep = ctx.decrypt(sk, res)
    ref = ost.plain_stats(x)["cv"]
    assert np.sign(v[0]) == np.sign(mu) and abs(v[0] / ref - 1) < TOL, (v[0], ref)
    _, rp = ctx.decrypt(sk, ctx.query(evk, "cv", col, opts=opts))
    assert rep["depth_used"] == rp["depth_used"] + 1
    if (k, t) == (7, 3):
        assert rep["depth_used"] == 18


@pytest.mark.parametrize("n", [2048, 3000])
def test_pcc_parity_small(deep, n):
    from oracle import stats as ost
    ctx, sk, evk, oc, ok = deep
    x, y = workloads.pcc_pair(n, seed=6)
    ox, cx = shared_column(deep, x, 31)
    oy, cy = shared_column(deep, y, 32)
    res = ctx.query(evk, "pcc", cx, cy, opts=dict(B_x=1.0, B_y=20.0, cheb_log2deg=5, newton_steps=2))
    want = ost.pcc(ost.CkksEv(oc, ok), ox, oy, n, 1.0, 20.0, 5, 2)
    check_same(ctx, res.cts()[0], want)
    v, _ = ctx.decrypt(sk, res)
    assert abs(v[0] / ost.plain_stats(x, y)["pcc"] - 1) < TOL


def test_query_batch_equals_single(deep):
    ctx, sk, evk, oc, ok = deep
    x = workloads.lognormal_column(1500, seed=8)
    x2, y2 = workloads.pcc_pair(2048, seed=9)
    cx = ctx.encrypt_column(evk, x, 41)
    c2 = ctx.encrypt_column(evk, x2, 42)
    cy = ctx.encrypt_column(evk, y2, 43)
    qs = [("kurt", cx, None, OPTS12), ("pcc", c2, cy, dict(OPTS12, B_x=1.0)), ("cv", cx, None, OPTS12)]
    batch = ctx.query_batch(evk, qs)
    for q, rb in zip(qs, batch):
        rs = ctx.query(evk, q[0], q[1], q[2], q[3])
        a = ctx.ct_export(rb.cts()[0])
        b = ctx.ct_export(rs.cts()[0])
        assert a[2:] == b[2:] and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_bad_query_arguments(deep):
    import paper_2508_12093_gb300 as pp
    ctx, sk, evk, oc, ok = deep
    cx = ctx.encrypt_column(evk, workloads.lognormal_column(100, seed=1), 1)
    with pytest.raises(pp.PpstError) as e:
        ctx.query(evk, "pcc", cx, None, OPTS12)
    assert e.value.code == -1
    with pytest.raises(pp.PpstError) as e:
        ctx.query(evk, "kurt", cx, None, dict(OPTS12, cheb_log2deg=10))  # depth 22 > 19 levels
    assert e.value.code == -2
    with pytest.raises(pp.PpstError) as e:
        ctx.query(evk, "kurt", cx, None, dict(OPTS12, newton_steps=-1))
    assert e.value.code == -1


# ---------------------------------------------------------------------------
# N = 2^16
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(workloads.PARAMS["n16_d6"])
    sk, evk = ctx.keygen(2)
    return ctx, sk, evk


OPTS16 = dict(B_x=20.0, B_y=20.0, cheb_log2deg=7, newton_steps=3)


@pytest.mark.parametrize("stat", ["skew", "kurt", "cv"])
def test_statistics_full_size(big, stat):
    from oracle import stats as ost
    ctx, sk, evk = big
    x = workloads.lognormal_column(32768, seed=1)
    col = ctx.encrypt_column(evk, x, 3)
    v, rep = ctx.decrypt(sk, ctx.query(evk, stat, col, opts=OPTS16))
    ref = ost.plain_stats(x)[stat]
    assert abs(v[0] / ref - 1) < TOL, (v[0], ref)
    assert rep["level_out"] >= 0


@pytest.mark.parametrize("mu", [-4.0, 5.0])
def test_sign_aware_cv_full_size(big, mu):
    """N = 2^16: the sign-aware CV of a 32,768-row normal column with a negative
    or positive mean within 1e-3 of FP64; for the positive mean it agrees with
    the positive-mean CV."""
    from oracle import stats as ost
    ctx, sk, evk = big
    x = workloads.normal_column(32768, seed=3, mu=mu, sigma=3.0)
    col = ctx.encrypt_column(evk, x, 7)
    opts = dict(OPTS16, B_x=8.0)
    v, rep = ctx.decrypt(sk, ctx.query(evk, "cv_signed", col, opts=opts))
    ref = ost.plain_stats(x)["cv"]
    assert abs(v[0] / ref - 1) < TOL, (v[0], ref)
    assert rep["depth_used"] == 18
    if mu > 0:
        p, _ = ctx.decrypt(sk, ctx.query(evk, "cv", col, opts=opts))
        assert abs(p[0] / v[0] - 1) < TOL


def test_pcc_full_size(big):
    from oracle import stats as ost
    ctx, sk, evk = big
    x, y = workloads.pcc_pair(32768, seed=1)
    cx, cy = ctx.encrypt_column(evk, x, 3), ctx.encrypt_column(evk, y, 4)
    v, _ = ctx.decrypt(sk, ctx.query(evk, "pcc", cx, cy, opts=dict(OPTS16, B_x=1.0)))
    ref = ost.plain_stats(x, y)["pcc"]
    assert abs(v[0] / ref - 1) < TOL, (v[0], ref)


def test_multi_ciphertext_column_full_size(big):
    """A 100,000-row column (4 ciphertexts, ragged tail): Z-score and kurtosis."""
    from oracle import stats as ost
    ctx, sk, evk = big
    x = workloads.lognormal_column(100000, seed=2)
    col = ctx.encrypt_column(evk, x, 5)
    ref = ost.plain_stats(x)
    v, _ = ctx.decrypt(sk, ctx.query(evk, "kurt", col, opts=OPTS16))
    assert abs(v[0] / ref["kurt"] - 1) < TOL
    z, rep = ctx.decrypt(sk, ctx.query(evk, "zscore", col, opts=OPTS16))
    assert len(z) == 100000 and rep["n_cts"] == 4
    assert np.abs(z - ref["znorm"]).max() / np.abs(ref["znorm"]).max() < TOL


def test_million_row_columns_full_size(big):
    """The largest columns of the served workload: 1,000,000 rows (31 ciphertexts,
    ragged tail) for Z-score, CV and PCC, as one batch."""
    from oracle import stats as ost
    ctx, sk, evk = big
    n = 1_000_000
    x = workloads.lognormal_column(n, seed=4)
    b, y = workloads.pcc_pair(n, seed=5)
    cx, cb, cy = (ctx.encrypt_column(evk, v, 6 + i) for i, v in enumerate((x, b, y)))
    res = ctx.query_batch(evk, [("zscore", cx, None, OPTS16), ("cv", cx, None, OPTS16),
                                ("pcc", cb, cy, dict(OPTS16, B_x=1.0))])
    ref = ost.plain_stats(x)
    z, rep = ctx.decrypt(sk, res[0])
    assert len(z) == n and rep["n_cts"] == 31
    assert np.abs(z - ref["znorm"]).max() / np.abs(ref["znorm"]).max() < TOL
    v, _ = ctx.decrypt(sk, res[1])
    assert abs(v[0] / ref["cv"] - 1) < TOL
    v, _ = ctx.decrypt(sk, res[2])
    assert abs(v[0] / ost.plain_stats(b, y)["pcc"] - 1) < TOL


def test_constant_column_runs(big):
    """A constant column has variance 0, outside CryptoInvSqrt's domain (0, 2]: the
    result is meaningless but the query completes (domain errors cannot be seen
    on encrypted data)."""
    ctx, sk, evk = big
    col = ctx.encrypt_column(evk, np.full(5000, 3.0), 9)
    v, rep = ctx.decrypt(sk, ctx.query(evk, "kurt", col, opts=OPTS16))
    assert rep["depth_used"] == 19 and np.isfinite(v[0])


def test_batch_full_size(big):
    """Twelve mixed queries over six columns of uneven lengths (the batched
    workload's shape) as one batch: every result identical to the query run
    alone, and within 1e-3 of FP64."""
    from oracle import stats as ost
    ctx, sk, evk = big
    lens = workloads.log_uniform_lengths(6, 1024, 32768, seed=7)
    cols, data = [], []
    for i, n in enumerate(lens):
        if i % 2 == 0:
            x = workloads.lognormal_column(int(n), seed=10 + i)
            data.append((x, None))
            cols.append((ctx.encrypt_column(evk, x, 20 + i), None))
        else:
            x, y = workloads.pcc_pair(int(n), seed=10 + i)
            data.append((x, y))
            cols.append((ctx.encrypt_column(evk, x, 20 + i), ctx.encrypt_column(evk, y, 40 + i)))
    qs = []
    for (cx, cy), (x, y) in zip(cols, data):
        if cy is None:
            qs += [("skew", cx, None, OPTS16), ("kurt", cx, None, OPTS16)]
        else:
            qs += [("pcc", cx, cy, dict(OPTS16, B_x=1.0)), ("cv", cy, None, OPTS16)]
    batch = ctx.query_batch(evk, qs)
    for q, rb in zip(qs, batch):
        rs = ctx.query(evk, q[0], q[1], q[2], q[3])
        a, b = ctx.ct_export(rb.cts()[0]), ctx.ct_export(rs.cts()[0])
        assert a[2:] == b[2:] and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), q[0]
    for i, ((x, y), rb) in enumerate(zip([d for d in data for _ in range(2)], batch)):
        name = qs[i][0]
        ref = ost.plain_stats(y, None)["cv"] if name == "cv" else ost.plain_stats(x, y)[name]
        v, _ = ctx.decrypt(sk, rb)
        assert abs(v[0] / ref - 1) < TOL, (name, v[0], ref)


def test_hmult_full_size_matches_oracle():
    """HMult + key switch at N = 2^16, top level (24 limbs, dnum = 6): limbs
    bit-exact against the oracle on shared keys and ciphertexts."""
    import paper_2508_12093_gb300 as pp
    from oracle import ckks as ock
    prm = workloads.PARAMS["n16_d6"]
    ctx = pp.Context(prm)
    sk, evk = ctx.keygen(2, rotations=[1])
    oc = ock.Ckks(ock.Params(**prm))
    ok = oc.keygen(2, rotations=[1])
    for j in (0, 5):
        b, a = ctx.evk_export(evk, -1, j)
        assert np.array_equal(b, ok["relin"].b[j]) and np.array_equal(a, ok["relin"].a[j])
    x = workloads.lognormal_column(32768, seed=1)
    ox = oc.encrypt_column(ok["pk"], x, 3)[0]
    gx = ctx.ct_import(ox.c0, ox.c1, ox.level, ox.scale)
    c0, c1, lv, sc = ctx.ct_export(ctx.hmult(evk, gx, gx))
    want = oc.hmult(ox, ox, ok)
    assert (lv, sc) == (want.level, want.scale)
    assert np.array_equal(c0, want.c0) and np.array_equal(c1, want.c1)
    r0, r1, _, _ = ctx.ct_export(ctx.rotate(evk, gx, 1))
    rw = oc.rotate(ox, 1, ok)
    assert np.array_equal(r0, rw.c0) and np.array_equal(r1, rw.c1)
