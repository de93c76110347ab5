"""CryptoInvSqrt through the C ABI: bit-exact against the oracle at N = 2^12,
and the inverse-square-root accuracy sweep of Sec. 7.2 at N = 2^16 (16,384
points in [0.001, 1] and 16,384 in [1, 100], pre-normalised by B = 100)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

DEEP12 = dict(log_n=12, n_q=20, n_p=2, dnum=10, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)


@pytest.mark.parametrize("k,t", [(3, 1), (5, 2), (6, 0), (7, 3), (8, 2)])
def test_inv_sqrt_parity(k, t):
    import paper_2508_12093_gb300 as pp
    from oracle import ckks as ock
    from oracle import stats as ost
    ctx = pp.Context(DEEP12)
    sk, evk = ctx.keygen(5)
    oc = ock.Ckks(ock.Params(**DEEP12))
    ok = oc.keygen(5)
    v = workloads.uniform_column(oc.prm.S, seed=8, lo=0.05, hi=2.0)
    o = oc.encrypt_column(ok["pk"], v, 9)[0]
    g = ctx.ct_import(o.c0, o.c1, o.level, o.scale)
    want = ost.crypto_inv_sqrt(ost.CkksEv(oc, ok), o, 3.0, k, t)
    got = ctx.inv_sqrt(evk, g, 3.0, k, t)
    c0, c1, lv, sc = ctx.ct_export(got)
    assert (lv, sc) == (want.level, want.scale)
    assert np.array_equal(c0, want.c0) and np.array_equal(c1, want.c1)
    if t >= 2:
        y = ctx.decrypt_ct(sk, got)
        assert np.abs(y * np.sqrt(3.0 * v) - 1).max() < 1e-3


def test_inv_sqrt_arguments():
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(DEEP12)
    sk, evk = ctx.keygen(5)
    g = ctx.encrypt_ints(evk, np.zeros(ctx.N, dtype=np.int64), 1, 0, 2.0 ** 40)
    for args, code in (((1.0, 1, 1), -1), ((1.0, 5, 11), -1), ((-2.0, 5, 1), -1), ((1.0, 10, 6), -2)):
        with pytest.raises(pp.PpstError) as e:
            ctx.inv_sqrt(evk, g, *args)
        assert e.value.code == code


def test_inv_sqrt_sweep_sec72():
    """Mean relative error of 1/sqrt(x) over the Sec. 7.2 grid at N = 2^16 with the
    paper's own approximation settings (degree 2^9 - 1, 6 Newton steps: depth 22 of
    the 23 levels, no bootstrapping) and with the statistics' default (2^7 - 1, 3)."""
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(workloads.PARAMS["n16_d6"])
    sk, evk = ctx.keygen(2)
    x = workloads.inv_sqrt_grid()
    assert len(x) == ctx.S
    B = 100.0
    col = ctx.encrypt_column(evk, x / B, 3)
    ref = 1.0 / np.sqrt(x)
    mre = {}
    for k, t in ((9, 6), (7, 3)):
        y = ctx.decrypt_ct(sk, ctx.inv_sqrt(evk, col.cts()[0], B, k, t))
        mre[(k, t)] = float(np.mean(np.abs(y - ref) / ref))
    print("Sec. 7.2 grid MRE:", mre)
    assert mre[(9, 6)] < 1e-6        # the paper reports 5.08e-5 with bootstrapping (context)
    assert mre[(7, 3)] < 1e-4
