"""GPU parity of the evaluator ops, through the C ABI, against the oracle.

Every comparison is bit-exact on coefficient-domain limbs: both sides derive
their keys and noise from the same seeds (independent ChaCha20 streams) and
the GPU imports the oracle's ciphertexts (encoding is FP64 and not bit-exact
across two FFT implementations, so parity starts from shared ciphertexts).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

# N = 2^12, 6 Q primes (q0 60-bit, 40-bit), 2 special primes, 3 digits of 2
SMALL = dict(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)


@pytest.fixture(scope="module")
def env():
    import paper_2508_12093_gb300 as pp
    from oracle import ckks as ock
    ctx = pp.Context(SMALL)
    sk, evk = ctx.keygen(7)
    oc = ock.Ckks(ock.Params(**SMALL))
    ok = oc.keygen(7, rotations=[1 << i for i in range(SMALL["log_n"] - 1)])
    return ctx, sk, evk, oc, ok


def fresh(env, seed, lo=-1.0, hi=1.0):
    ctx, sk, evk, oc, ok = env
    x = workloads.uniform_column(oc.prm.S, seed=seed, lo=lo, hi=hi)
    o = oc.encrypt_column(ok["pk"], x, seed)[0]
    g = ctx.ct_import(o.c0, o.c1, o.level, o.scale)
    return x, o, g


def same(ctx, g, o):
    c0, c1, lv, sc = ctx.ct_export(g)
    assert lv == o.level, (lv, o.level)
    assert sc == o.scale, (sc, o.scale)
    assert np.array_equal(c0, o.c0), "c0 limbs differ"
    assert np.array_equal(c1, o.c1), "c1 limbs differ"


@pytest.mark.parametrize("name", ["toy12", "n16_d6", "n16_d3", "n16_d12"])
def test_prime_chain_matches_oracle(name):
    import paper_2508_12093_gb300 as pp
    from oracle import ckks as ock
    prm = workloads.PARAMS[name]
    ctx = pp.Context(prm)
    op = ock.Params(**prm)
    assert ctx.primes == op.q + op.p


def test_keys_match_oracle(env):
    ctx, sk, evk, oc, ok = env
    assert np.array_equal(ctx.sk_export(sk), ok["s"])
    for j in range(len(ok["relin"].b)):
        b, a = ctx.evk_export(evk, -1, j)
        assert np.array_equal(a, ok["relin"].a[j]) and np.array_equal(b, ok["relin"].b[j]), j
    for r in (1, 64, oc.prm.S // 2):
        b, a = ctx.evk_export(evk, r, 1)
        assert np.array_equal(a, ok["rot"][r].a[1]) and np.array_equal(b, ok["rot"][r].b[1]), r


def test_encryption_matches_oracle(env):
    ctx, sk, evk, oc, ok = env
    x = workloads.uniform_column(oc.prm.S, seed=4)
    m = oc.encode_ints(x, oc.prm.scale)
    g = ctx.encrypt_ints(evk, np.array(m, dtype=np.int64), 9, 2, oc.prm.scale)
    o = oc.encrypt_ints(ok["pk"], m, 9, 2)
    same(ctx, g, o)


def test_import_export_roundtrip(env):
    ctx = env[0]
    x, o, g = fresh(env, 11)
    same(ctx, g, o)
    d = ctx.drop(g, 2)
    same(ctx, d, env[3].drop(o, 2))


def test_elementwise_ops(env):
    ctx, sk, evk, oc, ok = env
    _, oa, ga = fresh(env, 12)
    _, ob, gb = fresh(env, 13)
    same(ctx, ctx.add(ga, gb), oc.add(oa, ob))
    same(ctx, ctx.sub(ga, gb), oc.sub(oa, ob))
    for c in (0.75, -1.0, 3.0e-9, 1e3):
        same(ctx, ctx.add_const(ga, c), oc.add_const(oa, c))
    for k in (2, -3, 12345, 0):
        same(ctx, ctx.mul_int(ga, k), oc.mul_int(oa, k))
    # mixed levels: the higher operand is dropped
    same(ctx, ctx.add(ctx.drop(ga, 3), gb), oc.add(oc.drop(oa, 3), ob))


def test_rescale_and_mul_const(env):
    ctx, sk, evk, oc, ok = env
    _, oa, ga = fresh(env, 14)
    same(ctx, ctx.rescale(ga), oc.rescale(oa))
    for c in (0.37, -1.5, 1.0 / 2048, 123.456, 1e-12):
        same(ctx, ctx.mul_const(ga, c), oc.mul_const(oa, c))
    tgt = oa.scale * (1 + 2.0 ** -25)
    same(ctx, ctx.mul_const(ga, 0.5, tgt), oc.mul_const(oa, 0.5, tgt))
    lo = oc.drop(oa, 1)
    same(ctx, ctx.mul_const(ctx.drop(ga, 1), 0.9), oc.mul_const(lo, 0.9))


def test_lin_comb(env):
    ctx, sk, evk, oc, ok = env
    xs, os_, gs = zip(*[fresh(env, 30 + i) for i in range(5)])
    # different scales: steer one operand first (same op on both sides)
    o1 = oc.mul_const(os_[1], 1.0, os_[1].scale * (1 + 2.0 ** -28))
    g1 = ctx.mul_const(gs[1], 1.0, gs[1].scale * (1 + 2.0 ** -28))
    lv = o1.level
    olist = [oc.drop(os_[0], lv), o1] + [oc.drop(o, lv) for o in os_[2:]]
    glist = [ctx.drop(gs[0], lv), g1] + [ctx.drop(g, lv) for g in gs[2:]]
    coeffs = [0.25, -3.5, 1e-3, 7.0, -0.125]
    for n in (1, 3, 5):
        same(ctx, ctx.lin_comb(glist[:n], coeffs[:n], 2.0 ** 40), oc.lin_comb(olist[:n], coeffs[:n], 2.0 ** 40))
    # more terms than one group of loads in flight (8), a ragged last group, the maximum (32)
    rng = np.random.default_rng(12)
    for n in (8, 9, 20, 32):
        idx = [k % 5 for k in range(n)]
        cs = list(rng.uniform(-4, 4, n))
        same(ctx, ctx.lin_comb([glist[k] for k in idx], cs, 2.0 ** 40),
             oc.lin_comb([olist[k] for k in idx], cs, 2.0 ** 40))


def test_hmult_all_levels(env):
    ctx, sk, evk, oc, ok = env
    xa, oa, ga = fresh(env, 15)
    xb, ob, gb = fresh(env, 16)
    for lv in range(oc.prm.L, 0, -1):
        o = oc.hmult(oc.drop(oa, lv), ob, ok)
        g = ctx.hmult(evk, ctx.drop(ga, lv), gb)
        same(ctx, g, o)
    # square (same operand twice) and decrypted value
    g = ctx.hmult(evk, ga, ga)
    same(ctx, g, oc.hmult(oa, oa, ok))
    assert np.abs(ctx.decrypt_ct(sk, g) - xa * xa).max() < 2.0 ** -20


def test_rotations(env):
    ctx, sk, evk, oc, ok = env
    xa, oa, ga = fresh(env, 17)
    for r in (1, 2, 64, oc.prm.S // 2):
        same(ctx, ctx.rotate(evk, ga, r), oc.rotate(oa, r, ok))
    low = oc.drop(oa, 2)
    same(ctx, ctx.rotate(evk, ctx.drop(ga, 2), 8), oc.rotate(low, 8, ok))
    rs = ctx.rotsum(evk, ga)
    same(ctx, rs, oc.rotsum(oa, ok))
    assert abs(ctx.decrypt_ct(sk, rs)[5] - xa.sum()) < 1e-5
    assert np.abs(ctx.decrypt_ct(sk, ctx.rotate(evk, ga, 3 * 0 + 16)) - np.roll(xa, -16)).max() < 1e-6


@pytest.mark.parametrize("log_n", [10, 11, 13, 14, 15, 16])
def test_every_ring_degree(log_n):
    """Transform pass shapes for every supported N: import/export round trip,
    HMult and one rotation, bit-exact against the oracle."""
    import paper_2508_12093_gb300 as pp
    from oracle import ckks as ock
    prm = dict(log_n=log_n, n_q=3, n_p=1, dnum=3, q0_bits=60, q_bits=45, p_bits=60, log_scale=45)
    ctx = pp.Context(prm)
    sk, evk = ctx.keygen(3, rotations=[1])
    oc = ock.Ckks(ock.Params(**prm))
    ok = oc.keygen(3, rotations=[1])
    x = workloads.uniform_column(oc.prm.S, seed=log_n)
    o = oc.encrypt_column(ok["pk"], x, 4)[0]
    g = ctx.ct_import(o.c0, o.c1, o.level, o.scale)
    same(ctx, g, o)
    same(ctx, ctx.hmult(evk, g, g), oc.hmult(o, o, ok))
    same(ctx, ctx.rotate(evk, g, 1), oc.rotate(o, 1, ok))


def test_error_codes(env):
    import paper_2508_12093_gb300 as pp
    ctx, sk, evk, oc, ok = env
    _, oa, ga = fresh(env, 18)
    low = ctx.drop(ga, 0)
    with pytest.raises(pp.PpstError) as e:
        ctx.hmult(evk, low, low)
    assert e.value.code == -2
    with pytest.raises(pp.PpstError) as e:
        ctx.mul_const(low, 2.0)
    assert e.value.code == -2
    with pytest.raises(pp.PpstError) as e:
        ctx.rotate(evk, ga, 3)             # no Galois key for 3
    assert e.value.code == -8
    other = ctx.mul_const(ga, 1.0, ga.scale * (1 + 2.0 ** -10))
    with pytest.raises(pp.PpstError) as e:
        ctx.add(ctx.drop(ga, other.level), other)
    assert e.value.code == -3
    with pytest.raises(pp.PpstError) as e:
        ctx.drop(ga, 9)
    assert e.value.code == -1
    with pytest.raises(pp.PpstError) as e:  # an empty column
        ctx.encrypt_column(evk, np.zeros(0), 1)
    assert e.value.code == -1
    with pytest.raises(pp.PpstError) as e:  # a non-finite value cannot be encoded
        ctx.encrypt_column(evk, np.array([1.0, np.nan]), 1)
    assert e.value.code == -1
    for bad in (dict(SMALL, log_n=9), dict(SMALL, n_q=1), dict(SMALL, dnum=7), dict(SMALL, n_p=17)):
        with pytest.raises(pp.PpstError) as e:
            pp.Context(bad)
        assert e.value.code == -1


@pytest.mark.parametrize("n_q,dnum", [(12, 1), (12, 2), (12, 3), (12, 4), (12, 6), (12, 12), (24, 2), (24, 3),
                                        (24, 4), (24, 6)])
def test_every_digit_count(n_q, dnum):
    """Key switching for every decomposition of a 12-prime chain (digits of
    12, 6, 4, 3, 2 and 1 primes, K = digit size) and of the 24-prime chain the
    autotuner chooses from (digits of 12, 8, 6, 4): HMult at the top level and
    one level down, and a rotation, bit-exact against the oracle."""
    import paper_2508_12093_gb300 as pp
    from oracle import ckks as ock
    prm = dict(log_n=12, n_q=n_q, n_p=n_q // dnum, dnum=dnum, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
    ctx = pp.Context(prm)
    sk, evk = ctx.keygen(11, rotations=[5])
    oc = ock.Ckks(ock.Params(**prm))
    ok = oc.keygen(11, rotations=[5])
    x = workloads.uniform_column(oc.prm.S, seed=3)
    o = oc.encrypt_column(ok["pk"], x, 4)[0]
    g = ctx.ct_import(o.c0, o.c1, o.level, o.scale)
    same(ctx, ctx.hmult(evk, g, g), oc.hmult(o, o, ok))
    same(ctx, ctx.hmult(evk, ctx.drop(g, 6), g), oc.hmult(oc.drop(o, 6), o, ok))
    same(ctx, ctx.rotate(evk, g, 5), oc.rotate(o, 5, ok))
    assert np.abs(ctx.decrypt_ct(sk, ctx.rotate(evk, g, 5)) - np.roll(x, -5)).max() < 1e-6


def test_bounded_wait_timeout_is_reported(env):
    """A kernel whose barrier wait runs out (nothing is copied; the wait is bounded
    by 20 ms) records the timeout in the error word and returns: the next
    synchronising call reports PPST_E_CUDA once, and the context stays usable."""
    import paper_2508_12093_gb300 as pp
    ctx, sk, evk, oc, ok = env
    ctx.selftest_wait(20000)
    with pytest.raises(pp.PpstError) as e:
        ctx.sync()
    assert e.value.code == -6
    ctx.sync()  # the word was cleared
    _, oa, ga = fresh(env, 19)
    same(ctx, ctx.hmult(evk, ga, ga), oc.hmult(oa, oa, ok))
    with pytest.raises(pp.PpstError) as e:
        ctx.selftest_wait(0)
    assert e.value.code == -1


@pytest.mark.parametrize("tile", [4, 8, 16])
def test_inner_product_tiles_agree(env, tile):
    """The inner product's tile (chunks per block) changes speed only: HMult and a
    rotation bit-exact against the oracle for every tile."""
    import paper_2508_12093_gb300 as pp
    ctx, sk, evk, oc, ok = env
    _, oa, ga = fresh(env, 23)
    ctx.set_tile(tile)
    try:
        same(ctx, ctx.hmult(evk, ga, ga), oc.hmult(oa, oa, ok))
        same(ctx, ctx.rotate(evk, ga, 4), oc.rotate(oa, 4, ok))
    finally:
        ctx.set_tile(4)
    with pytest.raises(pp.PpstError) as e:
        ctx.set_tile(5)
    assert e.value.code == -1


@pytest.mark.parametrize("min_blocks", [0, 1 << 20])
def test_pass_block_shapes_agree(env, min_blocks):
    """Every transform pass with 16 sub-transforms per block (0) or 4 (2^20), and
    the inner product's smallest tile: HMult at two levels, a rotation and a
    rotate-and-sum bit-exact against the oracle."""
    import paper_2508_12093_gb300 as pp
    ctx, sk, evk, oc, ok = env
    _, oa, ga = fresh(env, 24)
    _, ob, gb = fresh(env, 25)
    ctx.set_pass_blocks(min_blocks)
    try:
        same(ctx, ctx.hmult(evk, ga, gb), oc.hmult(oa, ob, ok))
        same(ctx, ctx.hmult(evk, ctx.drop(ga, 2), gb), oc.hmult(oc.drop(oa, 2), ob, ok))
        same(ctx, ctx.rotate(evk, ga, 4), oc.rotate(oa, 4, ok))
        same(ctx, ctx.rotsum(evk, ga), oc.rotsum(oa, ok))
        same(ctx, ctx.mul_const(ga, 0.37), oc.mul_const(oa, 0.37))
    finally:
        ctx.set_pass_blocks(228)
    with pytest.raises(pp.PpstError) as e:
        ctx.set_pass_blocks((1 << 20) + 1)
    assert e.value.code == -1
