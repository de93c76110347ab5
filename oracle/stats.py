"""Statistic programs of PP-STAT over an evaluator, plus FP64 references.

TEST INFRASTRUCTURE (oracle). The schedules here follow the paper:

* CryptoInvSqrt (Sec. 5, Alg. 2 with n = 2, Alg. 3, Eq. 1 and Eq. 3): the
  input v in (0, 2] is shifted to u = v - 1 (Eq. 1), a degree 2^k - 1
  Chebyshev interpolant of F(u, C) = 1 / (sqrt(C) sqrt(u + 1)) gives the
  initial guess (Alg. 3; no bootstrapping here), then t Newton steps
  y <- 1.5 y - x' y^3 with x' = v * C / 2 (Alg. 2 with the constant C of
  Eq. 3 folded into the 1/n multiplier).
* CryptoSqrt (Eq. 4): the Chebyshev interpolant of sqrt(C) sqrt(u + 1) alone.
* Mean(x, B) and Variance(x, B) with the pre-normalisation constants folded
  into the plaintext multipliers (Sec. 6.1, Eq. 2).
* ZNorm (Alg. 4), Kurt (Alg. 5), Skew (Sec. 6: mirrors Alg. 5 with the third
  moment), CV (Alg. 6 for a positive mean, without Sign), the sign-aware CV
  (Alg. 6 with Sign read as mu * CryptoInvSqrt(mu^2)), PCC (Sec. 6.5).

Readings where the paper is silent (the same on the GPU side):
* Chebyshev evaluation is baby-step giant-step in the Chebyshev basis with
  T_{2i} = 2 T_i^2 - 1, T_{2i+1} = 2 T_i T_{i+1} - T_1, giant steps T_{2^m}
  and recursive division p = q T_n + r; a leaf sum sum_i c_i T_i is one
  linear combination with integer weights round(c_i q_l) and a single rescale,
  its scale steered to a target so every Add sees equal scales.
* Newton's three products are associated as (x' y)(y y): same products as
  Alg. 2, depth 2 per step instead of 3.
* Columns longer than one ciphertext are summed before one rotate-and-sum;
  the centred sums of skewness, kurtosis and PCC, consumed only by their final
  product, are dropped to that product's level before being reduced;
  padding slots are zero and their contribution to the centred moments
  ((-mu)^p per pad) is subtracted with integer multiples of mu^p.
"""
import math

import numpy as np

# ---------------------------------------------------------------------------
# Chebyshev interpolation (Sec. 3.4, Eq. 1, Eq. 3, Eq. 4)
# ---------------------------------------------------------------------------


def inv_sqrt_target(C):
    """Eq. 3 with B -> C: F(u, C) = 1 / (sqrt(C) * sqrt(u + 1)), 0 for u <= -1."""
    def F(u):
        return 1.0 / (math.sqrt(C) * math.sqrt(u + 1.0)) if u > -1.0 else 0.0
    return F


def sqrt_target(C):
    """Eq. 4 with B -> C: F(u, C) = sqrt(C) * sqrt(u + 1), 0 for u < -1."""
    def F(u):
        return math.sqrt(C) * math.sqrt(u + 1.0) if u >= -1.0 else 0.0
    return F


def cheb_coeffs(F, d):
    """Interpolant of F at the d+1 Chebyshev nodes of the first kind:
    c_k = (2/(d+1)) sum_j F(cos th_j) cos(k th_j), th_j = pi (j + 1/2)/(d+1),
    with c_0 halved, so that p(x) = sum_k c_k T_k(x). FP64, in this order."""
    n = d + 1
    th = [math.pi * (j + 0.5) / n for j in range(n)]
    f = [F(math.cos(t)) for t in th]
    c = []
    for k in range(n):
        s = 0.0
        for j in range(n):
            s += f[j] * math.cos(k * th[j])
        c.append(2.0 * s / n)
    c[0] *= 0.5
    return c


def cheb_split(c):
    """Chebyshev-basis division by T_n, n = len(c)/2:  p = q T_n + r with
    q_0 = c_n, q_i = 2 c_{n+i}, r_0 = c_0, r_i = c_i - c_{2n-i}  (from
    T_{n+i} = 2 T_n T_i - T_{n-i})."""
    n = len(c) // 2
    q = [c[n]] + [2.0 * c[n + i] for i in range(1, n)]
    r = [c[0]] + [c[i] - c[2 * n - i] for i in range(1, n)]
    return q, r


def cheb_eval(ev, u, c):
    """Evaluate sum_k c_k T_k(u) (len(c) = 2^k) by baby-step giant-step."""
    k = len(c).bit_length() - 1
    assert 1 << k == len(c) and k >= 1
    b = (k + 1) // 2
    T = {1: u}
    for i in range(2, (1 << b) + 1):
        if i % 2 == 0:
            h = T[i // 2]
            T[i] = ev.add_const(ev.mul_int(ev.hmult(h, h), 2), -1.0)
        else:
            p = ev.mul_int(ev.hmult(T[(i - 1) // 2], T[(i + 1) // 2]), 2)
            t1 = ev.mul_const(ev.drop(T[1], ev.level(p) + 1), 1.0, ev.scale(p))
            T[i] = ev.sub(p, t1)
    for m in range(b + 1, k):
        h = T[1 << (m - 1)]
        T[1 << m] = ev.add_const(ev.mul_int(ev.hmult(h, h), 2), -1.0)
    return _cheb_rec(ev, T, c, 1 << b, ev.nominal_scale())


def _rec_level(ev, T, length, baby):
    """Level at which _cheb_rec returns for a coefficient list of `length`."""
    if length <= baby:
        return min(ev.level(T[i]) for i in range(1, length)) - 1
    n = length // 2
    lq = min(_rec_level(ev, T, n, baby), ev.level(T[n])) - 1
    return min(lq, _rec_level(ev, T, n, baby))


def _cheb_rec(ev, T, c, baby, target):
    if len(c) <= baby:
        lv = min(ev.level(T[i]) for i in range(1, len(c)))
        acc = ev.lin_comb([ev.drop(T[i], lv) for i in range(1, len(c))], c[1:], target)
        return ev.add_const(acc, c[0])
    n = len(c) // 2
    q, r = cheb_split(c)
    lvl = min(_rec_level(ev, T, n, baby), ev.level(T[n]))
    ql = ev.prime(lvl)
    tq = target * float(ql) / ev.scale(T[n])
    prod = ev.hmult(_cheb_rec(ev, T, q, baby, tq), T[n])
    rest = _cheb_rec(ev, T, r, baby, ev.scale(prod))
    return ev.add(prod, rest)


# ---------------------------------------------------------------------------
# CryptoInvSqrt / CryptoSqrt (Sec. 5, Alg. 2, Alg. 3, Eq. 3, Eq. 4)
# ---------------------------------------------------------------------------

def crypto_inv_sqrt(ev, v, C, k, t):
    """approx 1/sqrt(C * v) for v in (0, 2]: Chebyshev guess + t Newton steps."""
    c = cheb_coeffs(inv_sqrt_target(C), (1 << k) - 1)
    y = cheb_eval(ev, ev.add_const(v, -1.0), c)
    xh = ev.mul_const(v, C / 2.0)
    for _ in range(t):
        y2 = ev.hmult(y, y)
        xy = ev.hmult(xh, y)
        b = ev.hmult(xy, y2)
        a = ev.mul_const(ev.drop(y, ev.level(b) + 1), 1.5, ev.scale(b))
        y = ev.sub(a, b)
    return y


def crypto_sqrt(ev, v, C, k):
    """approx sqrt(C * v) for v in (0, 2]: the Chebyshev interpolant of Eq. 4."""
    c = cheb_coeffs(sqrt_target(C), (1 << k) - 1)
    return cheb_eval(ev, ev.add_const(v, -1.0), c)


# ---------------------------------------------------------------------------
# Mean, Variance and the five statistics (Sec. 6)
# ---------------------------------------------------------------------------

def col_sum(ev, cts):
    acc = cts[0]
    for ct in cts[1:]:
        acc = ev.add(acc, ct)
    return acc


def variance(ev, cts, n, B, R):
    """Variance(x, B) = sum (x_i / (B sqrt n))^2 - (sum x_i / (B n))^2 = Var / B^2,
    depth 2 (Sec. 6.1); R = rotate-and-sum of the column, shared with Mean."""
    c = 1.0 / (B * math.sqrt(n))
    acc = None
    for ct in cts:
        y = ev.mul_const(ct, c)
        z = ev.hmult(y, y)
        acc = z if acc is None else ev.add(acc, z)
    a = ev.rotsum(acc)
    m = ev.mul_const(R, 1.0 / (B * n))
    return ev.sub(a, ev.hmult(m, m))


def _centred_power_terms(ev, cts, mu, power):
    """sum over the column's ciphertexts of (x - mu)^power, slot by slot (not
    yet reduced over the slots)."""
    acc = None
    for ct in cts:
        x1 = ev.sub(ct, mu)
        x2 = ev.hmult(x1, x1)
        xp = ev.hmult(x2, x2) if power == 4 else ev.hmult(x2, x1)
        acc = xp if acc is None else ev.add(acc, xp)
    return acc


def _rotsum_at(ev, a, level):
    """Rotate-and-sum of `a` after dropping it to `level` (never above its own).
    Sec. 6.1 leaves open at which level the sums are reduced; a sum whose value
    is consumed only by a product many levels lower is dropped to that level
    first, so its rotations switch keys over fewer limbs."""
    return ev.rotsum(ev.drop(a, min(level, ev.level(a))))


def znorm(ev, cts, n, B, k, t):
    """Alg. 4: (x - Mean(x)) * CryptoInvSqrt(Variance(x, B), B^2); one output
    ciphertext per input ciphertext."""
    R = ev.rotsum(col_sum(ev, cts))
    mu = ev.mul_const(R, 1.0 / n)
    inv = crypto_inv_sqrt(ev, variance(ev, cts, n, B, R), B * B, k, t)
    return [ev.hmult(ev.sub(ct, mu), inv) for ct in cts]


def kurt(ev, cts, n, B, k, t):
    """Alg. 5: Mean((x - mu)^4) * CryptoInvSqrt(Variance(x, B), B^2)^4 (plain,
    not excess, kurtosis)."""
    R = ev.rotsum(col_sum(ev, cts))
    mu = ev.mul_const(R, 1.0 / n)
    S4 = _centred_power_terms(ev, cts, mu, 4)
    inv = crypto_inv_sqrt(ev, variance(ev, cts, n, B, R), B * B, k, t)
    inv2 = ev.hmult(inv, inv)
    inv4 = ev.hmult(inv2, inv2)
    X = _rotsum_at(ev, S4, ev.level(inv4) + 1)
    pads = len(cts) * ev.slots() - n
    if pads:
        mu2 = ev.hmult(mu, mu)
        X = ev.sub(X, ev.mul_int(ev.hmult(mu2, mu2), pads))
    num = ev.mul_const(X, 1.0 / n)
    return ev.hmult(num, inv4)


def skew(ev, cts, n, B, k, t):
    """Skewness, the third-moment mirror of Alg. 5 (Sec. 6 omits it):
    Mean((x - mu)^3) * CryptoInvSqrt(Variance(x, B), B^2)^3."""
    R = ev.rotsum(col_sum(ev, cts))
    mu = ev.mul_const(R, 1.0 / n)
    S3 = _centred_power_terms(ev, cts, mu, 3)
    inv = crypto_inv_sqrt(ev, variance(ev, cts, n, B, R), B * B, k, t)
    inv3 = ev.hmult(ev.hmult(inv, inv), inv)
    X = _rotsum_at(ev, S3, ev.level(inv3) + 1)
    pads = len(cts) * ev.slots() - n
    if pads:
        mu2 = ev.hmult(mu, mu)
        X = ev.add(X, ev.mul_int(ev.hmult(mu2, mu), pads))
    num = ev.mul_const(X, 1.0 / n)
    return ev.hmult(num, inv3)


def cv(ev, cts, n, B, k, t):
    """Alg. 6 for a positive mean (no Sign): CryptoSqrt(Variance(x, B), B^2) *
    CryptoInvSqrt(Mean(x, B), B)^2."""
    R = ev.rotsum(col_sum(ev, cts))
    muB = ev.mul_const(R, 1.0 / (B * n))
    isq = crypto_inv_sqrt(ev, muB, B, k, t)
    mu_inv = ev.hmult(isq, isq)
    std = crypto_sqrt(ev, variance(ev, cts, n, B, R), B * B, k)
    return ev.hmult(std, mu_inv)


def cv_signed(ev, cts, n, B, k, t):
    """Alg. 6 with its Sign, for a mean of either sign: CV = Std(x) * (1 / |mu|) *
    sign(mu). Sign(mu) is mu * CryptoInvSqrt(mu^2, B^2) = mu / |mu| (the identity
    sign(x) = x / sqrt(x^2) on the inverse root that the method already has), and
    the inverse of the sign-corrected mean, CryptoInvSqrt(mu * sign(mu), B)^2 =
    1 / |mu|, is that same CryptoInvSqrt(mu^2, B^2): one inverse-root chain of the
    mean in place of Alg. 6's Sign (a depth-32 minimax polynomial) followed by a
    second chain. The input (mu / B)^2 lies in (0, 1] for |mu| <= B; Alg. 6's line
    order is kept: tmp = Std * mu_inv, then CV = tmp * sign."""
    R = ev.rotsum(col_sum(ev, cts))
    mu = ev.mul_const(R, 1.0 / n)
    muB = ev.mul_const(R, 1.0 / (B * n))
    mu_inv = crypto_inv_sqrt(ev, ev.hmult(muB, muB), B * B, k, t)   # 1 / |mu|
    sign = ev.hmult(mu, mu_inv)
    std = crypto_sqrt(ev, variance(ev, cts, n, B, R), B * B, k)
    return ev.hmult(ev.hmult(std, mu_inv), sign)


def pcc(ev, xcts, ycts, n, Bx, By, k, t):
    """Sec. 6.5:Cov(x, y) * CryptoInvSqrt(Var(x,Bx),Bx^2) * CryptoInvSqrt(Var(y,By),By^2)."""
    Rx = ev.rotsum(col_sum(ev, xcts))
    Ry = ev.rotsum(col_sum(ev, ycts))
    mux = ev.mul_const(Rx, 1.0 / n)
    muy = ev.mul_const(Ry, 1.0 / n)
    acc = None
    for xc, yc in zip(xcts, ycts):
        p = ev.hmult(ev.sub(xc, mux), ev.sub(yc, muy))
        acc = p if acc is None else ev.add(acc, p)
    ix = crypto_inv_sqrt(ev, variance(ev, xcts, n, Bx, Rx), Bx * Bx, k, t)
    iy = crypto_inv_sqrt(ev, variance(ev, ycts, n, By, Ry), By * By, k, t)
    Cs = _rotsum_at(ev, acc, min(ev.level(ix), ev.level(iy)) + 1)
    pads = len(xcts) * ev.slots() - n
    if pads:
        Cs = ev.sub(Cs, ev.mul_int(ev.hmult(mux, muy), pads))
    cov = ev.mul_const(Cs, 1.0 / n)
    return ev.hmult(ev.hmult(cov, ix), iy)


# ---------------------------------------------------------------------------
# evaluators
# ---------------------------------------------------------------------------

class CkksEv:
    """The exact oracle evaluator (oracle.ckks.Ckks + evaluation keys)."""

    def __init__(self, ckks, keys):
        self.c, self.keys = ckks, keys
        self.trace = None       # optional list collecting every op output

    def _t(self, ct):
        if self.trace is not None:
            self.trace.append(ct)
        return ct

    def level(self, ct):
        return ct.level

    def scale(self, ct):
        return ct.scale

    def prime(self, level):
        return self.c.primes[level]

    def nominal_scale(self):
        return self.c.prm.scale

    def slots(self):
        return self.c.prm.S

    def add(self, a, b):
        return self._t(self.c.add(a, b))

    def sub(self, a, b):
        return self._t(self.c.sub(a, b))

    def add_const(self, a, x):
        return self._t(self.c.add_const(a, x))

    def mul_int(self, a, k):
        return self._t(self.c.mul_int(a, k))

    def mul_const(self, a, x, target=None):
        return self._t(self.c.mul_const(a, x, target))

    def lin_comb(self, cts, coeffs, target):
        return self._t(self.c.lin_comb(cts, coeffs, target))

    def hmult(self, a, b):
        return self._t(self.c.hmult(a, b, self.keys))

    def drop(self, a, level):
        return self.c.drop(a, level)

    def rotsum(self, a):
        return self._t(self.c.rotsum(a, self.keys))


class SimCt:
    """Noise-free FP64 stand-in for a ciphertext: slot values, level and scale
    bookkeeping exactly as the CKKS evaluator tracks them."""

    def __init__(self, v, level, scale):
        self.v, self.level, self.scale = np.asarray(v, dtype=np.float64), level, float(scale)


class SimEv:
    """Runs a schedule on FP64 slot vectors with the same level/scale rules:
    the algorithmic error of Chebyshev + Newton without CKKS noise."""

    def __init__(self, primes, nominal_scale, slots):
        self.primes, self.s0, self.S = list(primes), float(nominal_scale), slots

    def encrypt(self, x, level=None):
        v = np.zeros(self.S)
        v[:len(x)] = x
        return SimCt(v, len(self.primes) - 1 if level is None else level, self.s0)

    def level(self, ct):
        return ct.level

    def scale(self, ct):
        return ct.scale

    def prime(self, level):
        return self.primes[level]

    def nominal_scale(self):
        return self.s0

    def slots(self):
        return self.S

    def _need(self, lv):
        if lv < 0:
            raise ValueError("depth exhausted")

    def add(self, a, b):
        return SimCt(a.v + b.v, min(a.level, b.level), a.scale)

    def sub(self, a, b):
        return SimCt(a.v - b.v, min(a.level, b.level), a.scale)

    def add_const(self, a, x):
        return SimCt(a.v + x, a.level, a.scale)

    def mul_int(self, a, k):
        return SimCt(a.v * k, a.level, a.scale)

    def mul_const(self, a, x, target=None):
        self._need(a.level - 1)
        return SimCt(a.v * x, a.level - 1, a.scale if target is None else target)

    def lin_comb(self, cts, coeffs, target):
        lv = cts[0].level
        assert all(c.level == lv for c in cts)
        self._need(lv - 1)
        v = np.zeros(self.S)
        for ct, x in zip(cts, coeffs):
            v = v + ct.v * x
        return SimCt(v, lv - 1, target)

    def hmult(self, a, b):
        lv = min(a.level, b.level)
        self._need(lv - 1)
        return SimCt(a.v * b.v, lv - 1, a.scale * b.scale / self.primes[lv])

    def drop(self, a, level):
        return SimCt(a.v, level, a.scale)

    def rotsum(self, a):
        return SimCt(np.full(self.S, math.fsum(a.v)), a.level, a.scale)


# ---------------------------------------------------------------------------
# FP64 plaintext statistics (population moments; two passes, exact sums)
# ---------------------------------------------------------------------------

def plain_stats(x, y=None):
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    mu = math.fsum(x) / n
    d = x - mu
    m2 = math.fsum(d * d) / n
    m3 = math.fsum(d * d * d) / n
    m4 = math.fsum(d * d * d * d) / n
    out = {"mean": mu, "var": m2, "znorm": d / math.sqrt(m2), "skew": m3 / m2 ** 1.5,
           "kurt": m4 / (m2 * m2), "cv": math.sqrt(m2) / mu}
    if y is not None:
        y = np.asarray(y, dtype=np.float64)
        my = math.fsum(y) / n
        e = y - my
        out["pcc"] = math.fsum(d * e) / math.sqrt(math.fsum(d * d) * math.fsum(e * e))
    return out
