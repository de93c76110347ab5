"""Pins for the oracle's exact arithmetic: primes, transform, RNS, PRNG.

Every check here compares the oracle with something other than itself:
schoolbook products, Python big integers, sympy's primality test, the RFC 8439
test vector, algebraic identities that a wrong index or sign would break.
"""
import math
import random

import numpy as np
import pytest

from conftest import read_golden
from oracle import ckks
from oracle._clib import lib, ptr32, ptr64

CFG1 = dict(log_n=12, n_q=12, n_p=1, dnum=12, q0_bits=60, q_bits=40, p_bits=60, log_scale=40)
CFG2 = dict(log_n=16, n_q=24, n_p=4, dnum=6, q0_bits=60, q_bits=50, p_bits=60, log_scale=50)


# ---------------------------------------------------------------------------
# primes
# ---------------------------------------------------------------------------

def test_is_prime_matches_sympy():
    sympy = pytest.importorskip("sympy")
    rng = random.Random(5)
    cands = [rng.getrandbits(64) | 1 for _ in range(300)]
    cands += [2, 3, 4, 561, 1105, 2 ** 61 - 1, 2 ** 64 - 59, 3825123056546413051]  # carmichaels, strong pseudoprime
    for n in cands:
        assert bool(lib.or_is_prime(n)) == bool(sympy.isprime(n)), n


@pytest.mark.parametrize("cfg", [CFG1, CFG2])
def test_prime_chain_rule(cfg):
    sympy = pytest.importorskip("sympy")
    p = ckks.Params(**cfg)
    M = 2 * p.N
    allp = p.q + p.p
    assert len(set(allp)) == len(allp)
    for q in allp:
        assert sympy.isprime(q) and q % M == 1
    # q0: largest prime = 1 mod 2N below 2^q0_bits
    q0 = p.q[0]
    assert q0 < 2 ** cfg["q0_bits"]
    assert not any(sympy.isprime(c) for c in range(q0 + M, 2 ** cfg["q0_bits"], M))
    # middle primes alternate above / below 2^q_bits and are the nearest ones
    B = 2 ** cfg["q_bits"]
    above = [q for q in p.q[1:] if q > B]
    below = [q for q in p.q[1:] if q < B]
    assert p.q[1::2] == above and p.q[2::2] == below
    assert not any(sympy.isprime(c) for c in range(B + 1, max(above), M) if c not in above)
    assert not any(sympy.isprime(c) for c in range(min(below), B, M) if c not in below)


def test_cfg2_modulus_size_matches_paper_scale():
    # the paper's logPQ = 1443 bits (Sec. 7.1); this chain: 60 + 23*50 + 4*60
    p = ckks.Params(**CFG2)
    logpq = sum(math.log2(q) for q in p.q + p.p)
    assert abs(logpq - 1450) < 0.01
    assert logpq < 1772  # 128-bit bound for N = 2^16, ternary secret (HE standard)


# ---------------------------------------------------------------------------
# negacyclic transform
# ---------------------------------------------------------------------------

def schoolbook_negacyclic(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += a[i] * b[j]
            else:
                out[k - N] -= a[i] * b[j]
    return [v % q for v in out]


@pytest.mark.parametrize("log_n", [2, 3, 4, 5, 6])
def test_poly_mul_matches_schoolbook(log_n):
    N = 1 << log_n
    prm = ckks.Params(log_n=max(log_n, 2), n_q=3, n_p=1, dnum=3, q0_bits=60, q_bits=50, p_bits=61, log_scale=40)
    c = ckks.Ckks(prm)
    rng = random.Random(log_n)
    idx = list(range(len(c.primes)))
    for trial in range(3):
        a = np.empty((len(idx), N), dtype=np.uint64)
        b = np.empty_like(a)
        for r, t in enumerate(idx):
            q = c.primes[t]
            if trial == 0:      # edge values
                a[r] = [q - 1] * N
                b[r] = [(q - 1) if i % 2 else 0 for i in range(N)]
            else:
                a[r] = [rng.randrange(q) for _ in range(N)]
                b[r] = [rng.randrange(q) for _ in range(N)]
        got = c.polymul(a, b, idx)
        for r, t in enumerate(idx):
            want = schoolbook_negacyclic([int(v) for v in a[r]], [int(v) for v in b[r]], c.primes[t])
            assert [int(v) for v in got[r]] == want


def test_transform_is_evaluation_at_odd_powers():
    prm = ckks.Params(log_n=4, n_q=2, n_p=1, dnum=2, q0_bits=60, q_bits=50, p_bits=61, log_scale=40)
    c = ckks.Ckks(prm)
    N = prm.N
    q, psi = c.primes[1], c.psi[1]
    assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1
    rng = random.Random(1)
    a = [rng.randrange(q) for _ in range(N)]
    got = c.ntt(np.array([a], dtype=np.uint64), [1])[0]
    for k in range(N):
        assert int(got[k]) == sum(a[i] * pow(psi, (2 * k + 1) * i, q) for i in range(N)) % q
    back = c.intt(got[None, :], [1])[0]
    assert [int(v) for v in back] == a


# ---------------------------------------------------------------------------
# RNS: CRT, base conversion, ModDown, rescale, automorphism
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small():
    prm = ckks.Params(log_n=5, n_q=6, n_p=2, dnum=3, q0_bits=60, q_bits=50, p_bits=60, log_scale=50)
    return ckks.Ckks(prm)


def test_crt_reconstructs_big_integers(small):
    c = small
    idx = list(range(4))
    Q = math.prod(c.primes[t] for t in idx)
    rng = random.Random(2)
    vals = [rng.randrange(-(Q // 2), Q // 2) for _ in range(c.N)]
    vals[0], vals[1] = Q // 2, -(Q // 2) + 1
    rns = c.to_rns(vals, idx)
    assert c.crt_centred(rns, idx) == vals


def test_bconv_is_x_plus_small_multiple_of_Q(small):
    c = small
    src, dst = [1, 2, 3], [0, 4, 5, 6, 7]
    Q = math.prod(c.primes[t] for t in src)
    rng = random.Random(3)
    xs = [rng.randrange(Q) for _ in range(c.N)]
    xs[0], xs[1] = 0, Q - 1
    out = c.bconv(c.to_rns(xs, src), src, dst)
    for col, x in enumerate(xs):
        # the integer the conversion stands for, from its definition:
        # y = sum_i [x (Q/q_i)^-1]_{q_i} (Q/q_i) = x + u Q with 0 <= u < len(src)
        y = sum(((x * pow(Q // c.primes[i], -1, c.primes[i])) % c.primes[i]) * (Q // c.primes[i]) for i in src)
        u, rem = divmod(y - x, Q)
        assert rem == 0 and 0 <= u < len(src)
        for r, t in enumerate(dst):
            assert int(out[r, col]) == y % c.primes[t]


def test_mod_down_divides_multiples_of_P_exactly(small):
    c = small
    lv = 3
    ext = c.ext_index(lv)
    P = c.prm.P
    Q = math.prod(c.primes[t] for t in range(lv + 1))
    rng = random.Random(4)
    xs = [rng.randrange(-(Q // 2), Q // 2) for _ in range(c.N)]
    u = c.to_rns([P * x for x in xs], ext)
    got = c.mod_down(u, lv)
    assert c.crt_centred(got, list(range(lv + 1))) == xs


def test_mod_down_rounds_close_to_division(small):
    c = small
    lv = 2
    ext = c.ext_index(lv)
    P = c.prm.P
    QP = math.prod(c.primes[t] for t in ext)
    rng = random.Random(6)
    xs = [rng.randrange(-(QP // 2), QP // 2) for _ in range(c.N)]
    got = c.crt_centred(c.mod_down(c.to_rns(xs, ext), lv), list(range(lv + 1)))
    Q = math.prod(c.primes[t] for t in range(lv + 1))
    for x, y in zip(xs, got):
        # fast conversion without correction: y = (x - [x]_P - u P) / P
        # = floor(x / P) - u  (mod Q)  with 0 <= u < K
        d = (x // P - y) % Q
        assert 0 <= d < c.prm.K


def test_rescale_is_exact_rounding(small):
    c = small
    lv = 4
    idx = list(range(lv + 1))
    Q = math.prod(c.primes[t] for t in idx)
    ql = c.primes[lv]
    rng = random.Random(7)
    vals0 = [rng.randrange(-(Q // 2), Q // 2) for _ in range(c.N)]
    vals1 = [ql * rng.randrange(-100, 100) + (ql - 1) // 2 for _ in range(c.N)]   # near-tie edge
    ct = ckks.Ct(c.to_rns(vals0, idx), c.to_rns(vals1, idx), lv, 2.0 ** 50)
    out = c.rescale(ct)
    for vals, got in ((vals0, out.c0), (vals1, out.c1)):
        rec = c.crt_centred(got, idx[:-1])
        for v, r in zip(vals, rec):
            # round(v / ql), exact (ql odd: no ties)
            want = (2 * v + ql) // (2 * ql)
            assert r == want
    assert out.level == lv - 1 and out.scale == 2.0 ** 50 / ql


def test_automorphism_is_a_ring_homomorphism(small):
    c = small
    idx = [0, 1]
    rng = random.Random(8)
    a = np.array([[rng.randrange(c.primes[t]) for _ in range(c.N)] for t in idx], dtype=np.uint64)
    b = np.array([[rng.randrange(c.primes[t]) for _ in range(c.N)] for t in idx], dtype=np.uint64)
    for g in (5, 25, 2 * c.N - 1, 3):
        lhs = c.automorph(c.polymul(a, b, idx), g, idx)
        rhs = c.polymul(c.automorph(a, g, idx), c.automorph(b, g, idx), idx)
        assert np.array_equal(lhs, rhs)
    # composition and identity
    assert np.array_equal(c.automorph(c.automorph(a, 5, idx), 25, idx), c.automorph(a, 125, idx))
    assert np.array_equal(c.automorph(a, 1, idx), a)
    # X -> X^g sends the monomial X to X^g exactly
    mono = np.zeros((1, c.N), dtype=np.uint64)
    mono[0, 1] = 1
    img = c.automorph(mono, 2 * c.N - 1, [0])      # X -> X^(2N-1) = -X^(N-1)
    assert int(img[0, c.N - 1]) == c.primes[0] - 1 and int(img[0].sum()) == c.primes[0] - 1


# ---------------------------------------------------------------------------
# ChaCha20, SplitMix64 and the samplers
# ---------------------------------------------------------------------------

def test_chacha20_block_rfc8439_vector():
    rows, _ = read_golden("chacha20_block_rfc8439_2_3_2.txt")
    key = np.array([int(w, 16) for w in rows["key"]], dtype=np.uint32)
    nonce = np.array([int(w, 16) for w in rows["nonce"]], dtype=np.uint32)
    out = np.zeros(16, dtype=np.uint32)
    lib.or_chacha20_block(ptr32(key), int(rows["counter"][0]), ptr32(nonce), ptr32(out))
    assert [int(v) for v in out] == [int(w, 16) for w in rows["out"]]


def test_splitmix64_reference_outputs():
    import ctypes
    _, lines = read_golden("splitmix64_seed0.txt")
    st = ctypes.c_uint64(0)
    got = [lib.or_splitmix64(ctypes.byref(st)) for _ in range(3)]
    assert got == [int(h, 16) for h in lines]


def test_sampler_distributions():
    prm = ckks.Params(log_n=14, n_q=2, n_p=1, dnum=2, q0_bits=60, q_bits=50, p_bits=60, log_scale=50)
    c = ckks.Ckks(prm)
    s = c.sample_ternary(9, 1, 0)
    counts = [(s == v).mean() for v in (-1, 0, 1)]
    assert all(abs(f - 1 / 3) < 0.02 for f in counts)
    e = c.sample_gauss(9, 3, 0)
    assert abs(e.mean()) < 0.1 and abs(e.std() - 3.2) < 0.1 and np.abs(e).max() <= 19
    u = c.sample_uniform(9, 2, 0, [1])[0]
    q = c.primes[1]
    assert int(u.max()) < q and abs(float(u.mean()) / q - 0.5) < 0.02
    # different nonces give different streams; same inputs give the same stream
    assert not np.array_equal(c.sample_ternary(9, 1, 0), c.sample_ternary(9, 1, 1))
    assert np.array_equal(c.sample_gauss(9, 3, 0), e)


def test_cdt_table_matches_gaussian_mass():
    T = np.zeros(19, dtype=np.uint64)
    lib.or_cdt_table(3.2, 19, ptr64(T))
    w = [math.exp(-x * x / (2 * 3.2 ** 2)) for x in range(20)]
    tot = w[0] + 2 * sum(w[1:])
    for k in range(19):
        p = (w[0] + 2 * sum(w[1:k + 1])) / tot
        assert abs(int(T[k]) / 2 ** 64 - p) < 1e-12
    assert all(int(T[k]) < int(T[k + 1]) for k in range(18))
