"""Seeded synthetic workloads and parameter-set descriptors.

This module only draws input data (numpy generators) and names parameter
sets; it holds none of the method's arithmetic, so both the GPU library's
tests/benchmark and the CPU oracle can take their inputs from it.

The paper's datasets (UCI Adult, Medical Cost Insurance; Sec. 7.4) are not
available; these stand-ins have the shapes the paper describes:
* insurance-like charges: lognormal(mu=9, sigma=0.9), scaled by 1/1000 as the
  paper scales `charges` before encryption (Sec. 7.4.2);
* a binary attribute (smoker-like) x ~ Bernoulli(0.2) and a charge-like
  y = lognormal(9, 0.6) + 20000 x + N(0, 3000^2), also scaled by 1/1000;
* uniform [0, 1) columns (toy case), uniform [0, 100] / [0, 20] (Sec. 7.3);
* normal columns with a negative mean (Sec. 6.4: the mean in CV's
  denominator may be negative);
* the inverse-square-root grid of Sec. 7.2: 16,384 points evenly spaced in
  [0.001, 1] and 16,384 in [1, 100].
"""
import numpy as np

# parameter sets: ring degree, prime counts and sizes, digit count, scale
PARAMS = {
    # N = 2^12 toy set: q0 60 bits, 11 x 40-bit primes, one 60-bit special
    # prime, one prime per digit, scale 2^40 (depth 11 = the Z-score depth)
    "toy12": dict(log_n=12, n_q=12, n_p=1, dnum=12, q0_bits=60, q_bits=40, p_bits=60, log_scale=40),
    # N = 2^16: q0 60 bits, 23 x 50-bit primes, K special 60-bit primes,
    # scale 2^50; K = alpha = 24 / dnum
    "n16_d6": dict(log_n=16, n_q=24, n_p=4, dnum=6, q0_bits=60, q_bits=50, p_bits=60, log_scale=50),
    "n16_d3": dict(log_n=16, n_q=24, n_p=8, dnum=3, q0_bits=60, q_bits=50, p_bits=60, log_scale=50),
    "n16_d4": dict(log_n=16, n_q=24, n_p=6, dnum=4, q0_bits=60, q_bits=50, p_bits=60, log_scale=50),
    "n16_d12": dict(log_n=16, n_q=24, n_p=2, dnum=12, q0_bits=60, q_bits=50, p_bits=60, log_scale=50),
}

SEEDS = dict(data=1, key=2, enc=3, arrival=4)


def uniform_column(n, seed=SEEDS["data"], lo=0.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, n)


def lognormal_column(n, seed=SEEDS["data"], mu=9.0, sigma=0.9, scale=1e-3):
    return np.random.default_rng(seed).lognormal(mu, sigma, n) * scale


def normal_column(n, seed=SEEDS["data"], mu=-4.0, sigma=2.0):
    """Normal values whose mean may be negative (the sign-aware CV's input)."""
    return np.random.default_rng(seed).normal(mu, sigma, n)


def pcc_pair(n, seed=SEEDS["data"], p=0.2, scale=1e-3):
    rng = np.random.default_rng(seed)
    x = (rng.random(n) < p).astype(np.float64)
    y = (rng.lognormal(9.0, 0.6, n) + 20000.0 * x + rng.normal(0.0, 3000.0, n)) * scale
    return x, y


def log_uniform_lengths(count, lo, hi, seed=SEEDS["data"]):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), count)).astype(np.int64)


def poisson_arrivals(count, rate_per_s, seed=SEEDS["arrival"]):
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


def inv_sqrt_grid():
    """Sec. 7.2: 16,384 points in [0.001, 1] and 16,384 in [1, 100]."""
    return np.concatenate([np.linspace(0.001, 1.0, 16384), np.linspace(1.0, 100.0, 16384)])
