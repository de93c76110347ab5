"""Pins for the oracle's CKKS layer and statistic programs.

Encode/decode are checked against direct evaluation of the polynomial at the
slot roots; homomorphic ops against plaintext arithmetic within noise bounds;
the Chebyshev / Newton code against numpy's Chebyshev routines and the closed
form 1/sqrt(x); the statistics against scipy.stats on the same data.
"""
import math

import numpy as np
import pytest

from oracle import ckks, stats
import workloads


@pytest.fixture(scope="module")
def toy():
    # N = 2^10, 6 Q primes, 2 special primes, 3 digits
    prm = ckks.Params(log_n=10, n_q=6, n_p=2, dnum=3, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
    c = ckks.Ckks(prm)
    keys = c.keygen(11, rotations=[1 << i for i in range(prm.log_n - 1)])
    return c, keys


def slot_roots(N):
    M = 2 * N
    e, v = [], 1
    for _ in range(N // 2):
        e.append(v)
        v = v * 5 % M
    return np.exp(1j * np.pi * np.array(e) / N)


def test_encode_evaluates_to_slots(toy):
    c, _ = toy
    rng = np.random.default_rng(0)
    z = rng.uniform(-3, 3, c.prm.S)
    m = np.array(c.encode_ints(z, 2.0 ** 40), dtype=np.float64)
    # the defining property: m(zeta^(5^j)) = Delta z_j (up to rounding of m)
    roots = slot_roots(c.N)
    vals = np.array([np.polynomial.polynomial.polyval(r, m) for r in roots[:64]])
    assert np.abs(vals.real / 2.0 ** 40 - z[:64]).max() < 1e-9
    assert np.abs(vals.imag / 2.0 ** 40).max() < 1e-9
    back = c.decode_ints(c.encode_ints(z, 2.0 ** 40), 2.0 ** 40)
    assert np.abs(back - z).max() / np.abs(z).max() < 2.0 ** -30


def test_decode_of_monomial_is_closed_form(toy):
    c, _ = toy
    for i in (0, 1, 7, c.N - 1):
        ints = [0] * c.N
        ints[i] = 3 * 2 ** 40
        got = c.decode_ints(ints, 2.0 ** 40)
        want = 3 * slot_roots(c.N) ** i
        assert np.abs(got - want.real).max() < 1e-10


def test_encrypt_decrypt_noise_bound(toy):
    c, keys = toy
    x = np.random.default_rng(1).uniform(-1, 1, c.prm.S)
    ct = c.encrypt_column(keys["pk"], x, 5)[0]
    m = c.decrypt_ints(keys["s"], ct)
    want = c.encode_ints(x, c.prm.scale)
    err = max(abs(a - b) for a, b in zip(m, want))
    # e = u e_pk + e0 + e1 s: |e| <= N (19) + 19 + N (19) for ternary u, s
    assert err <= 19 * (2 * c.N + 1)
    assert err > 0


def test_homomorphic_ops_match_plaintext(toy):
    c, keys = toy
    S = c.prm.S
    rng = np.random.default_rng(2)
    x, y = rng.uniform(-1, 1, S), rng.uniform(-1, 1, S)
    cx = c.encrypt_column(keys["pk"], x, 6)[0]
    cy = c.encrypt_column(keys["pk"], y, 7)[0]
    dec = lambda ct: c.decrypt(keys["s"], ct)
    tol = 2.0 ** -22    # fresh noise ~ 2^-26 at scale 2^40, N = 2^10
    assert np.abs(dec(c.add(cx, cy)) - (x + y)).max() < tol
    assert np.abs(dec(c.sub(cx, cy)) - (x - y)).max() < tol
    assert np.abs(dec(c.add_const(cx, 0.75)) - (x + 0.75)).max() < tol
    assert np.abs(dec(c.mul_int(cx, -3)) - (-3 * x)).max() < tol
    m = c.hmult(cx, cy, keys)
    assert m.level == c.prm.L - 1
    assert np.abs(dec(m) - x * y).max() < tol
    mc = c.mul_const(cx, -0.3)
    assert mc.scale == cx.scale and mc.level == cx.level - 1
    assert np.abs(dec(mc) + 0.3 * x).max() < tol
    for r in (1, 8, S // 2):
        assert np.abs(dec(c.rotate(cx, r, keys)) - np.roll(x, -r)).max() < tol
    assert np.abs(dec(c.rotsum(cx, keys)) - x.sum()).max() < 2.0 ** -20
    # lower levels: drop, then multiply
    d = c.hmult(c.drop(cx, 2), cy, keys)
    assert d.level == 1 and np.abs(dec(d) - x * y).max() < tol


def test_lin_comb(toy):
    c, keys = toy
    rng = np.random.default_rng(9)
    xs = [rng.uniform(-1, 1, c.prm.S) for _ in range(3)]
    cts = [c.encrypt_column(keys["pk"], x, 20 + i)[0] for i, x in enumerate(xs)]
    cts[1] = c.mul_const(c.drop(cts[1], cts[1].level), 1.0, cts[1].scale * (1 + 2.0 ** -30))
    lv = min(ct.level for ct in cts)
    cts = [c.drop(ct, lv) for ct in cts]
    # one term: exactly Mul(P) with the same target
    one = c.lin_comb([cts[0]], [0.3], cts[0].scale)
    ref = c.mul_const(cts[0], 0.3, cts[0].scale)
    assert np.array_equal(one.c0, ref.c0) and np.array_equal(one.c1, ref.c1) and one.scale == ref.scale
    # several terms at different scales: the weighted sum, at the target scale
    coeffs = [0.5, -1.25, 2.0]
    out = c.lin_comb(cts, coeffs, 2.0 ** 40)
    assert out.scale == 2.0 ** 40 and out.level == lv - 1
    want = sum(k * x for k, x in zip(coeffs, xs))
    assert np.abs(c.decrypt(keys["s"], out) - want).max() < 2.0 ** -20


def test_key_switch_changes_key(toy):
    c, keys = toy
    # switching the plain polynomial d (as c1 of (0, d)) under the relin key
    # gives (k0, k1) with k0 + k1 s = d s^2 + small
    prm = c.prm
    lv = prm.L
    idx = list(range(lv + 1))
    rng = np.random.default_rng(3)
    d = np.array([rng.integers(0, c.primes[t], c.N, dtype=np.uint64) for t in idx])
    k0, k1 = c.key_switch(d, keys["relin"], lv)
    s = c.to_rns(keys["s"], idx)
    lhs = c.vadd(k0, c.polymul(k1, s, idx), idx)
    rhs = c.polymul(d, c.polymul(s, s, idx), idx)
    diff = c.crt_centred(c.vsub(lhs, rhs, idx), idx)
    assert max(abs(v) for v in diff) < 2 ** 30     # tiny next to Q ~ 2^260


def test_depth_and_scale_errors(toy):
    c, keys = toy
    ct = c.encrypt_column(keys["pk"], [0.5], 8)[0]
    low = c.drop(ct, 0)
    with pytest.raises(ckks.DepthError):
        c.hmult(low, low, keys)
    with pytest.raises(ckks.DepthError):
        c.mul_const(low, 2.0)
    other = ckks.Ct(ct.c0, ct.c1, ct.level, ct.scale * (1 + 2.0 ** -10))
    with pytest.raises(ckks.ScaleError):
        c.add(ct, other)


# ---------------------------------------------------------------------------
# Chebyshev + Newton
# ---------------------------------------------------------------------------

def test_chebyshev_interpolates_at_nodes():
    for k in (3, 5, 7):
        d = (1 << k) - 1
        F = stats.inv_sqrt_target(4.0)
        c = stats.cheb_coeffs(F, d)
        nodes = np.cos(np.pi * (np.arange(d + 1) + 0.5) / (d + 1))
        got = np.polynomial.chebyshev.chebval(nodes, c)
        assert np.abs(got - np.array([F(x) for x in nodes])).max() < 1e-11


def test_chebyshev_error_decreases_with_degree():
    xs = np.linspace(-0.95, 1.0, 2001)
    F = stats.sqrt_target(9.0)
    errs = []
    for k in range(2, 10):
        c = stats.cheb_coeffs(F, (1 << k) - 1)
        errs.append(np.abs(np.polynomial.chebyshev.chebval(xs, c) - 3 * np.sqrt(xs + 1)).max())
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_cheb_split_identity():
    rng = np.random.default_rng(4)
    c = list(rng.normal(size=16))
    q, r = stats.cheb_split(c)
    Tn = [0.0] * 8 + [1.0]
    prod = np.polynomial.chebyshev.chebmul(q, Tn)
    rec = np.polynomial.chebyshev.chebadd(prod, r)
    assert np.allclose(rec[:16], c, atol=1e-12) and np.allclose(rec[16:], 0, atol=1e-12)


def sim_for(S=64, levels=40):
    primes = [2 ** 50 + 2 * i + 1 for i in range(levels)]     # only levels matter here
    return stats.SimEv(primes, 2.0 ** 50, S)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 7])
def test_bsgs_schedule_equals_chebval(k):
    ev = sim_for()
    u = np.linspace(-0.99, 0.99, 64)
    c = list(np.random.default_rng(k).normal(size=1 << k))
    got = stats.cheb_eval(ev, ev.encrypt(u), c)
    assert np.allclose(got.v, np.polynomial.chebyshev.chebval(u, c), rtol=1e-10, atol=1e-10)
    # depth k + 1 for k >= 3 (k for k = 2: a single baby step)
    assert ev.encrypt(u).level - got.level == (k + 1 if k >= 3 else k)


def test_newton_converges_to_closed_form():
    ev = sim_for(S=512)
    v = np.linspace(0.02, 2.0, 512)
    for C in (1.0, 400.0):
        y = stats.crypto_inv_sqrt(ev, ev.encrypt(v), C, 7, 3)
        assert np.abs(y.v * np.sqrt(C * v) - 1).max() < 1e-6
    # one Newton step on the exact root is a fixed point; from y0 the update is
    # 0.5 y (3 - x y^2)  (Alg. 1)
    y0 = np.full(512, 0.9)
    yv = 0.5 * y0 * (3 - v * y0 ** 2)
    assert np.allclose(1.5 * y0 - (v / 2) * y0 ** 3, yv)


def test_newton_basin_on_grid():
    # the Chebyshev guess y0 must lie in Newton's basin 0 < v y0^2 < 3 on (0, 2]
    v = np.linspace(1e-3, 2.0, 20001)
    for k in (3, 5, 7):
        for C in (0.0841, 1.0, 400.0):
            c = stats.cheb_coeffs(stats.inv_sqrt_target(C), (1 << k) - 1)
            y0 = np.polynomial.chebyshev.chebval(v - 1, c)
            r = C * v * y0 ** 2
            assert (r > 0).all() and (r < 3).all(), (k, C)


def test_inverse_by_squaring():
    ev = sim_for(S=128)
    v = np.linspace(0.05, 2.0, 128)
    y = stats.crypto_inv_sqrt(ev, ev.encrypt(v), 1.0, 7, 3)
    sq = ev.hmult(y, y)
    assert np.abs(sq.v * v - 1).max() < 1e-6


# ---------------------------------------------------------------------------
# statistics
# ---------------------------------------------------------------------------

def test_plain_stats_match_scipy():
    sp = pytest.importorskip("scipy.stats")
    x, y = workloads.pcc_pair(4096, seed=1)
    ref = stats.plain_stats(x, y)
    assert math.isclose(ref["skew"], sp.skew(x), rel_tol=1e-10)
    assert math.isclose(ref["kurt"], sp.kurtosis(x, fisher=False), rel_tol=1e-10)
    assert math.isclose(ref["pcc"], sp.pearsonr(x, y)[0], rel_tol=1e-10)
    assert np.allclose(ref["znorm"], sp.zscore(x), rtol=1e-10)
    assert math.isclose(ref["cv"], sp.variation(x), rel_tol=1e-10)


def test_scaled_mean_and_variance():
    ev = sim_for(S=1024)
    x = workloads.lognormal_column(1000, seed=2)
    ct = ev.encrypt(x)
    R = ev.rotsum(ct)
    B = 20.0
    v = stats.variance(ev, [ct], 1000, B, R)
    ref = stats.plain_stats(x)
    assert math.isclose(v.v[0], ref["var"] / B ** 2, rel_tol=1e-12)
    m = ev.mul_const(R, 1.0 / (B * 1000))
    assert math.isclose(m.v[0], ref["mean"] / B, rel_tol=1e-12)
    assert ct.level - v.level == 2       # Sec. 6.1: depth 2 before the inverse root


@pytest.mark.parametrize("n,nct", [(1000, 1), (1024, 1), (3000, 3)])
def test_statistics_schedules_simulated(n, nct):
    S = 1024
    ev = sim_for(S=S, levels=24)
    x, y = workloads.pcc_pair(n, seed=3)
    xl = workloads.lognormal_column(n, seed=4)
    ref_x = stats.plain_stats(xl)
    ref_p = stats.plain_stats(x, y)
    cts = [ev.encrypt(xl[i * S:(i + 1) * S]) for i in range(nct)]
    for name, f in (("skew", stats.skew), ("kurt", stats.kurt), ("cv", stats.cv)):
        r = f(ev, cts, n, 20.0, 7, 3)
        assert abs(r.v[0] / ref_x[name] - 1) < 1e-4, name
    z = stats.znorm(ev, cts, n, 20.0, 7, 3)
    zz = np.concatenate([c.v for c in z])[:n]
    assert np.abs(zz - ref_x["znorm"]).max() / np.abs(ref_x["znorm"]).max() < 1e-4
    xc = [ev.encrypt(x[i * S:(i + 1) * S]) for i in range(nct)]
    yc = [ev.encrypt(y[i * S:(i + 1) * S]) for i in range(nct)]
    r = stats.pcc(ev, xc, yc, n, 1.0, 20.0, 7, 3)
    assert abs(r.v[0] / ref_p["pcc"] - 1) < 1e-4


@pytest.mark.parametrize("mu", [-4.0, -1.5, 3.0])
def test_sign_aware_cv_simulated(mu):
    """Alg. 6 with Sign, through the noise-free simulator, on normal columns of
    either sign (3000 rows over three ciphertexts): the result is Std / mu,
    negative for a negative mean, within 1e-4 of scipy's variation; negating the
    column negates the result exactly (Sign flips, 1/|mu| and Std do not); for a
    positive mean it agrees with the positive-mean CV; it costs one level more
    than that CV (18 of 23 at degree 127 + 3 Newton steps)."""
    sp = pytest.importorskip("scipy.stats")
    S, n, B = 1024, 3000, 8.0
    ev = sim_for(S=S, levels=24)
    x = workloads.normal_column(n, seed=5, mu=mu, sigma=2.0)
    cts = [ev.encrypt(x[i * S:(i + 1) * S]) for i in range(3)]
    neg = [ev.encrypt(-x[i * S:(i + 1) * S]) for i in range(3)]
    r = stats.cv_signed(ev, cts, n, B, 7, 3)
    ref = sp.variation(x)
    assert math.copysign(1.0, ref) == math.copysign(1.0, mu)
    assert abs(r.v[0] / ref - 1) < 1e-4
    assert stats.cv_signed(ev, neg, n, B, 7, 3).v[0] == -r.v[0]
    assert cts[0].level - r.level == 18
    if mu > 0:
        p = stats.cv(ev, cts, n, B, 7, 3)
        assert abs(p.v[0] / r.v[0] - 1) < 1e-4 and cts[0].level - p.level == 17


def test_sign_aware_cv_on_ckks():
    """The sign-aware CV on the exact CKKS oracle (N = 2^12, 15 Q primes: the
    depth 14 of degree 31 + 2 Newton steps) for a negative-mean column spread
    over two ciphertexts with a ragged tail: negative, within 1e-3 of FP64, and
    the schedule ends at level 0."""
    prm = ckks.Params(log_n=12, n_q=15, n_p=1, dnum=15, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
    c = ckks.Ckks(prm)
    keys = c.keygen(2, rotations=[1 << i for i in range(prm.log_n - 1)])
    n = prm.S + 700
    x = workloads.normal_column(n, seed=8, mu=-3.0, sigma=3.0)
    cts = c.encrypt_column(keys["pk"], x, 5)
    r = stats.cv_signed(stats.CkksEv(c, keys), cts, n, 6.0, 5, 2)
    assert r.level == 0
    got = c.decrypt(keys["s"], r)[0]
    ref = stats.plain_stats(x)["cv"]
    assert ref < 0 and abs(got / ref - 1) < 1e-3


def test_znorm_on_ckks_cfg1_shape():
    """Full Z-score schedule on the exact CKKS oracle, N = 2^12, 12 Q primes
    (depth 11), within 1e-3 of FP64 plaintext."""
    prm = ckks.Params(log_n=12, n_q=12, n_p=1, dnum=12, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
    c = ckks.Ckks(prm)
    keys = c.keygen(2, rotations=[1 << i for i in range(prm.log_n - 1)])
    x = workloads.uniform_column(prm.S, seed=1)
    cts = c.encrypt_column(keys["pk"], x, 3)
    z = stats.znorm(stats.CkksEv(c, keys), cts, prm.S, 0.29, 3, 2)[0]
    assert z.level == 0
    got = c.decrypt(keys["s"], z)
    ref = stats.plain_stats(x)["znorm"]
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-3


@pytest.mark.slow
def test_kurtosis_on_ckks_reduced_at_consumer_level():
    """Kurtosis on the exact CKKS oracle (N = 2^12, 20 Q primes, depth 19 at
    degree 127 + 3 Newton steps) with the centred fourth-power sum reduced at
    the level of its final product (level 2 here, not 16): the rotations at a
    low level still give the statistic within 1e-3 of FP64, and the schedule
    reaches level 0 exactly."""
    prm = ckks.Params(log_n=12, n_q=20, n_p=2, dnum=10, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
    c = ckks.Ckks(prm)
    keys = c.keygen(2, rotations=[1 << i for i in range(prm.log_n - 1)])
    n = prm.S + 301
    x = workloads.lognormal_column(n, seed=15)
    cts = c.encrypt_column(keys["pk"], x, 63)
    ev = stats.CkksEv(c, keys)
    levels = []
    rotsum = ev.rotsum
    ev.rotsum = lambda a: (levels.append(a.level), rotsum(a))[1]
    r = stats.kurt(ev, cts, n, 20.0, 7, 3)
    assert r.level == 0
    # Mean's sum at the top, Variance's two levels down, the fourth-power sum at
    # level 2 (the product with inv^4 at level 1 consumes it)
    assert sorted(levels) == [2, 17, 19]
    got = c.decrypt(keys["s"], r)[0]
    assert abs(got / stats.plain_stats(x)["kurt"] - 1) < 1e-3


def test_symmetric_column_has_zero_skew():
    """Data symmetric about its mean: the plain skewness is 0 and the simulated
    schedule's numerator (the centred third-moment sum) vanishes, so the
    encrypted skewness is 0 up to the approximation's absolute error."""
    S = 1024
    ev = sim_for(S=S, levels=24)
    half = workloads.lognormal_column(500, seed=7)
    x = np.concatenate([half, 2 * half.mean() - half])  # mirrored about the mean
    assert abs(stats.plain_stats(x)["skew"]) < 1e-12
    r = stats.skew(ev, [ev.encrypt(x)], len(x), 20.0, 7, 3)
    assert abs(r.v[0]) < 1e-9


def test_lognormal_moments_closed_form():
    """Large-sample sanity check of the population moments against the closed
    forms of lognormal(mu, sigma): skew = (e^s2 + 2) sqrt(e^s2 - 1), kurt =
    e^(4 s2) + 2 e^(3 s2) + 3 e^(2 s2) - 3, CV = sqrt(e^s2 - 1)."""
    s2 = 0.3 ** 2
    x = np.random.default_rng(11).lognormal(1.0, 0.3, 1_000_000)
    st = stats.plain_stats(x)
    assert abs(st["skew"] / ((math.exp(s2) + 2) * math.sqrt(math.exp(s2) - 1)) - 1) < 0.03
    assert abs(st["kurt"] / (math.exp(4 * s2) + 2 * math.exp(3 * s2) + 3 * math.exp(2 * s2) - 3) - 1) < 0.03
    assert abs(st["cv"] / math.sqrt(math.exp(s2) - 1) - 1) < 0.005


def test_constant_column_is_outside_the_domain():
    """A constant column has variance 0: 1/sqrt(Var) is undefined (the FP64
    reference flags it; on encrypted data it cannot be detected)."""
    with pytest.raises(ZeroDivisionError), np.errstate(divide="ignore", invalid="ignore"):
        stats.plain_stats(np.full(100, 3.0))


def test_sec72_grid_simulated():
    """The inverse-square-root sweep of Sec. 7.2 (16,384 points in [0.001, 1] and
    16,384 in [1, 100], pre-normalised by B = 100) through the noise-free
    simulator: the approximation error alone, against 1/sqrt(x). With the
    statistics' settings (degree 127, 3 Newton steps) the mean relative error is
    of the paper's order (5.08e-5 with bootstrapping); with the paper's own
    settings (degree 511, 6 steps) Newton converges to FP64 precision."""
    x = workloads.inv_sqrt_grid()
    assert len(x) == 32768 and x.min() == 0.001 and x.max() == 100.0
    ev = sim_for(S=32768, levels=24)
    ref = 1.0 / np.sqrt(x)
    mre = {}
    for k, t in ((7, 3), (9, 6)):
        y = stats.crypto_inv_sqrt(ev, ev.encrypt(x / 100.0), 100.0, k, t)
        mre[(k, t)] = float(np.mean(np.abs(y.v - ref) / ref))
    assert 1e-5 < mre[(7, 3)] < 5e-5
    assert mre[(9, 6)] < 1e-12
