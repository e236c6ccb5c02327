"""The oracle's AMP dynamics against its state evolution (a prediction that does not come from
running the iteration).

For y = Q beta + w with Q ~ Gin(m, n), entries N(0, 1/m), delta = m/n, beta_i ~ (1-eps)
delta_0 + eps N(0, 1), and w ~ N(0, s_w^2), AMP with soft threshold theta_k = 1.1 tau_k
tracks
    tau_0^2 = s_w^2 + eps / delta,
    tau_{k+1}^2 = s_w^2 + E[(eta(B + tau_k Z; 1.1 tau_k) - B)^2] / delta,
with ||z^k||^2 / m -> tau_k^2 and ||x^{k+1} - beta||^2 / n -> delta (tau_{k+1}^2 - s_w^2).
The expectation is computed by Gauss-Hermite quadrature.  A dropped Onsager term, a wrong
threshold or a transposed product moves the trajectory far off this curve.  HD (Algorithm 1)
and the dense direct simulation both follow it (Theorem 1).
"""
import numpy as np
import pytest

import synth
from oracle.direct import DirectState, ginibre
from oracle.dynamics import amp, soft_threshold
from oracle.hd import GinibreOracle

EPS, SW = 0.1, 0.1


def state_evolution(delta, iters, thr=1.1):
    z, wz = np.polynomial.hermite_e.hermegauss(120)
    wz = wz / wz.sum()
    b, wb = z, wz                      # N(0, 1) amplitudes of the nonzero entries

    def mse(tau):
        theta = thr * tau
        e0 = np.sum(wz * soft_threshold(tau * z, theta) ** 2)
        r = b[:, None] + tau * z[None, :]
        e1 = np.sum(wb[:, None] * wz[None, :] * (soft_threshold(r, theta) - b[:, None]) ** 2)
        return (1 - EPS) * e0 + EPS * e1

    tau2 = [SW ** 2 + EPS / delta]
    mses = []
    for _ in range(iters):
        e = mse(np.sqrt(tau2[-1]))
        mses.append(e)
        tau2.append(SW ** 2 + e / delta)
    return np.array(tau2), np.array(mses)


@pytest.mark.parametrize("kind", ["hd", "direct"])
def test_amp_follows_state_evolution(kind):
    n, m, T = 8000, 4000, 30
    beta = synth.bernoulli_gauss(n, 3, p_nonzero=EPS)
    w = synth.noise(m, 3, sigma=SW)
    if kind == "hd":
        st = GinibreOracle(m, n, T, 17, sigma=m ** -0.5)
    else:
        st = DirectState(ginibre(np.random.default_rng(17), m, n, m ** -0.5))
    xs, zs = amp(st, beta, w, T)
    iters = len(xs)
    tau2, mses = state_evolution(m / n, iters)
    emp_tau2 = np.array([np.dot(z, z) / m for z in zs])
    emp_mse = np.array([np.dot(x - beta, x - beta) / n for x in xs])
    assert iters == 15 and len(zs) == 15
    np.testing.assert_allclose(emp_tau2, tau2[:len(zs)], rtol=0.12)
    np.testing.assert_allclose(emp_mse, mses, rtol=0.15)
    # AMP converges well below the initial error (IST without the Onsager term does not in 15 iterations)
    assert emp_mse[-1] < 0.35 * emp_mse[0]
