"""Seeded synthetic inputs for the Householder Dice workloads.

This module only draws inputs (initial conditions, signals, noise, per-trial sizes) with
numpy's PCG64; it holds none of the method's arithmetic and is the one module that both
the CUDA path's callers (tests, bench) and the oracle use.  The random vectors g_t the
method itself draws are not made here: each side generates them from the Philox
definition.

Workloads (sizes as in the paper's experiments and the synthetic benchmark set):
  ginibre_tanh  Gin(n, n), entries N(0, 1/n), n = 1000, T = 10, all Q, x_1 ~ N(0, I)
  haar_sign     Haar(n), n = 10^6, T = 100, Q / Q^T alternating, x_1 ~ N(0, I), x_0 = 0
  amp_batch     4096 trials of Gin(m, n), m = n/2, n ~ U{1000..100000}, T = 30,
                beta* ~ Bernoulli(0.1) x N(0, 1), noise N(0, 0.1^2)
  ista_batch    64 trials of Gin(n, n), n = 200000, T = 50 ISTA iterations (101 products),
                beta* ~ 0.2 delta_0 + 0.8 N(0, 2^2) (Section 2.1), noise N(0, 0.1^2)
  haar_large    Haar(n), n = 2*10^7, T = 256, all Q, x_1 ~ N(0, I)
  lasso_ista    Gin(m, n), m = n/2, entries N(0, 1/m), n = 10^7, 50 ISTA iterations
                (101 products), beta* ~ 0.2 delta_0 + 0.8 N(0, 2^2), noise N(0, 0.1^2)
                (Section 2.1, the run the paper times)
  spectral      A = [I_n 0] Q, Q ~ Haar(2n), n = 10^5, xi ~ N(0, I_n), start x ~ N(0, I_n),
                100 power iterations (Section 2.2)
"""
import numpy as np


def rng(seed, *salt):
    return np.random.default_rng(np.random.SeedSequence([int(seed) & 0xFFFFFFFF, *salt]))


def x1(n, seed, trial=0, dtype=np.float64):
    """Initial condition x_1 ~ N(0, I_n), independent of Q (Section 3.2)."""
    return rng(seed, 1, trial).standard_normal(n).astype(dtype)


def bernoulli_gauss(n, seed, trial=0, p_nonzero=0.1, scale=1.0, dtype=np.float64):
    """Sparse signal: each entry nonzero with probability p_nonzero, then N(0, scale^2)."""
    g = rng(seed, 2, trial)
    mask = g.random(n) < p_nonzero
    return (mask * scale * g.standard_normal(n)).astype(dtype)


def noise(m, seed, trial=0, sigma=0.1, dtype=np.float64):
    return (sigma * rng(seed, 3, trial).standard_normal(m)).astype(dtype)


def batch_sizes(count, lo, hi, seed):
    """Per-trial dimensions n_i ~ U{lo..hi}, as int64."""
    return rng(seed, 4).integers(lo, hi + 1, size=count, dtype=np.int64)


WORKLOADS = {
    "ginibre_tanh": dict(ensemble="ginibre", m=1000, n=1000, T=10, sigma_scale="1/sqrt(n)",
                         schedule="all_q", dynamics="tanh"),
    "haar_sign": dict(ensemble="haar", m=10**6, n=10**6, T=100, schedule="alternating",
                      dynamics="sign_mem"),
    "amp_batch": dict(ensemble="ginibre", trials=4096, n_lo=1000, n_hi=100000, ratio=0.5, T=30),
    "ista_batch": dict(ensemble="ginibre", trials=64, n=200000, iters=50),
    "haar_large": dict(ensemble="haar", m=2 * 10**7, n=2 * 10**7, T=256, schedule="all_q",
                       dynamics="norm_tanh"),
}
