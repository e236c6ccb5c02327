"""ISTA on Householder Dice against ISTA on a dense Gaussian matrix (the paper's Fig. 1a
comparison, Section 2.1, at a small size; the paper prints no values, so the pin is the
agreement of the two, which Theorem 1 guarantees in law).

beta* ~ 0.2 delta_0 + 0.8 N(0, 2^2), w ~ N(0, 0.1^2), tau = 0.3, threshold lambda tau = 0.6
(the Fig. 1 caption: rho = 0.2, sigma_s = 2, sigma_w = 0.1, tau = 0.3, lambda = 2).  Two
shapes: Gin(n, n) with entries N(0, 1/n) (the differentiable workload's shape) and the
paper's own design Gin(m, n), m = floor(n/2), entries N(0, 1/m).  Per iteration, the mean
MSE over independent trials of the HD oracle and of direct simulation agree within 4
combined standard errors, and the final MSEs pass a two-sample KS test.
"""
import numpy as np
import torch
from scipy import stats

import synth
from dyn_util import ista_f, ista_schedule
from oracle.hd import GinibreOracle


def hd_curve(n, K, seed, trial):
    beta = torch.tensor(synth.bernoulli_gauss(n, seed, trial=trial, p_nonzero=0.8, scale=2.0))
    w = torch.tensor(synth.noise(n, seed, trial=trial, sigma=0.1))
    ora = GinibreOracle(n, n, 2 * K + 1, seed, trial=trial, sigma=n ** -0.5)
    f = ista_f(w)
    theta, tau = torch.full((K,), 0.6, dtype=torch.float64), torch.tensor(0.3, dtype=torch.float64)
    sched = ista_schedule(K)
    x, xprev, mse = beta, None, []
    for t in range(1, 2 * K + 2):
        y = ora.apply(x, sched[t - 1])
        x, xprev = f(t, y, x, xprev, theta, tau), x
        if t >= 3 and t % 2 == 1:
            mse.append(float(torch.sum((x - beta) ** 2) / n))
    return mse


def direct_curve(n, K, rng):
    beta = (rng.random(n) < 0.8) * 2.0 * rng.standard_normal(n)
    w = 0.1 * rng.standard_normal(n)
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    y = A @ beta + w
    x, mse = np.zeros(n), []
    for _ in range(K):
        v = x + 0.3 * (A.T @ (y - A @ x))
        x = np.sign(v) * np.maximum(np.abs(v) - 0.6, 0.0)
        mse.append(float(np.sum((x - beta) ** 2) / n))
    return mse


def test_ista_mse_curve_matches_direct_simulation():
    n, K, trials = 80, 8, 300
    hd = np.array([hd_curve(n, K, 17, i) for i in range(trials)])
    rng = np.random.default_rng(2024)
    dr = np.array([direct_curve(n, K, rng) for _ in range(trials)])
    se = np.sqrt(hd.var(axis=0, ddof=1) / trials + dr.var(axis=0, ddof=1) / trials)
    gap = np.abs(hd.mean(axis=0) - dr.mean(axis=0))
    assert (gap <= 4.0 * se).all(), (gap / se)
    assert stats.ks_2samp(hd[:, -1], dr[:, -1]).pvalue > 1e-3
    # the iteration makes progress (guards against a curve that is flat in both)
    assert hd.mean(axis=0)[-1] < 0.9 * hd.mean(axis=0)[0]


def hd_curve_paper(n, K, seed, trial):
    """Eq. ista on Gin(m, n), m = floor(n/2): y = Q beta* + w, then Q x^k and Q^T r^k."""
    m = n // 2
    beta = torch.tensor(synth.bernoulli_gauss(n, seed, trial=trial, p_nonzero=0.8, scale=2.0))
    w = torch.tensor(synth.noise(m, seed, trial=trial, sigma=0.1))
    ora = GinibreOracle(m, n, 2 * K + 1, seed, trial=trial, sigma=m ** -0.5)
    y = ora.apply(beta, False) + w
    x, mse = torch.zeros(n, dtype=torch.float64), []
    for _ in range(K):
        v = x + 0.3 * ora.apply(y - ora.apply(x, False), True)
        x = torch.sign(v) * torch.clamp(v.abs() - 0.6, min=0.0)
        mse.append(float(torch.sum((x - beta) ** 2) / n))
    return mse


def direct_curve_paper(n, K, rng):
    m = n // 2
    beta = (rng.random(n) < 0.8) * 2.0 * rng.standard_normal(n)
    w = 0.1 * rng.standard_normal(m)
    A = rng.standard_normal((m, n)) / np.sqrt(m)
    y = A @ beta + w
    x, mse = np.zeros(n), []
    for _ in range(K):
        v = x + 0.3 * (A.T @ (y - A @ x))
        x = np.sign(v) * np.maximum(np.abs(v) - 0.6, 0.0)
        mse.append(float(np.sum((x - beta) ** 2) / n))
    return mse


def test_ista_mse_curve_matches_direct_simulation_paper_design():
    n, K, trials = 101, 10, 300      # m = 50: floor(n/2) on an odd n
    hd = np.array([hd_curve_paper(n, K, 23, i) for i in range(trials)])
    rng = np.random.default_rng(2025)
    dr = np.array([direct_curve_paper(n, K, rng) for _ in range(trials)])
    se = np.sqrt(hd.var(axis=0, ddof=1) / trials + dr.var(axis=0, ddof=1) / trials)
    gap = np.abs(hd.mean(axis=0) - dr.mean(axis=0))
    assert (gap <= 4.0 * se).all(), (gap / se)
    assert stats.ks_2samp(hd[:, -1], dr[:, -1]).pvalue > 1e-3
    # progress from x^0 = 0, whose MSE is E beta*^2 = 0.8 * 2^2 (at m = n/2 with 80 %
    # nonzeros the curve dips and rises again, so the first iterate is no reference)
    assert hd.mean(axis=0)[-1] < 0.9 * 3.2
