"""The oracle's pathwise derivative (torch float64 autograd through Algorithms 1 and 2 with the
draws fixed) against central finite differences of the same oracle: gradients with respect
to the initial condition and to the parameters of f_t, for Haar and Ginibre, Q / Q^T
alternating, all Q and mixed schedules.  This pins the reference for the library's reverse
mode; a wrong derivative anywhere in the chain (reflector construction, sign factor, basis
vectors, output sums) fails it."""
import numpy as np
import pytest
import torch

from oracle.adjoint import trajectory
from oracle.hd import make_oracle

F64 = torch.float64


def f_theta(t, y, x, xprev, theta, beta):
    """x_{t+1} = tanh(theta_t y_t) + beta x_{t-1} (x_0 = 0): smooth, with per-step parameters."""
    v = torch.tanh(theta[t - 1] * y)
    return v if xprev is None else v + beta * xprev


def f_square(t, y, x, xprev, theta, beta):
    """x_{t+1} = tanh(theta_t y_t) + beta x_t (square matrices, any schedule)."""
    return torch.tanh(theta[t - 1] * y) + beta * x


CASES = [
    ("haar", 24, 24, 9, [t % 2 == 0 for t in range(1, 10)], f_theta),
    ("haar", 17, 17, 8, [False] * 8, f_square),
    ("ginibre", 14, 23, 10, [t % 2 == 0 for t in range(1, 11)], f_theta),
    ("ginibre", 19, 19, 9, [t in (2, 3, 6) for t in range(1, 10)], f_square),
]


def loss_and_grads(ens, m, n, T, sched, f, x1, theta, beta, c, sigma):
    x1 = x1.clone().requires_grad_(True)
    theta = theta.clone().requires_grad_(True)
    beta = beta.clone().requires_grad_(True)
    out = trajectory(ens, m, n, T, 11, sched, f, x1, (theta, beta), sigma=sigma)
    L = torch.dot(c, out)
    gx, gt, gb = torch.autograd.grad(L, (x1, theta, beta))
    return L.item(), gx, gt, gb


@pytest.mark.parametrize("ens,m,n,T,sched,f", CASES)
def test_oracle_gradient_matches_finite_differences(ens, m, n, T, sched, f):
    rng = np.random.default_rng(5)
    sigma = 1.0 if ens == "haar" else m ** -0.5
    n_in = m if sched[0] else n
    x1 = torch.tensor(rng.standard_normal(n_in), dtype=F64)
    theta = torch.tensor(0.6 + 0.4 * rng.random(T), dtype=F64)
    beta = torch.tensor(0.3, dtype=F64)
    with torch.no_grad():
        out = trajectory(ens, m, n, T, 11, sched, f, x1, (theta, beta), sigma=sigma)
    c = torch.tensor(rng.standard_normal(out.numel()), dtype=F64)
    _, gx, gt, gb = loss_and_grads(ens, m, n, T, sched, f, x1, theta, beta, c, sigma)

    def L(x1_, th_, b_):
        with torch.no_grad():
            return torch.dot(c, trajectory(ens, m, n, T, 11, sched, f, x1_, (th_, b_), sigma=sigma)).item()

    h = 1e-6
    for _ in range(3):   # random directions in x1
        v = torch.tensor(rng.standard_normal(n_in), dtype=F64)
        fd = (L(x1 + h * v, theta, beta) - L(x1 - h * v, theta, beta)) / (2 * h)
        assert abs(fd - torch.dot(gx, v).item()) <= 1e-6 * max(1.0, abs(fd)), (fd, torch.dot(gx, v).item())
    for j in (0, T // 2, T - 1):
        e = torch.zeros(T, dtype=F64)
        e[j] = 1.0
        fd = (L(x1, theta + h * e, beta) - L(x1, theta - h * e, beta)) / (2 * h)
        assert abs(fd - gt[j].item()) <= 1e-6 * max(1.0, abs(fd)), (j, fd, gt[j].item())
    fd = (L(x1, theta, beta + h) - L(x1, theta, beta - h)) / (2 * h)
    assert abs(fd - gb.item()) <= 1e-6 * max(1.0, abs(fd))


def test_haar_first_step_derivative_is_rank_one():
    """y_1 = ||x_1|| g / ||g|| (eq. H_1): dy_1/dx_1 = (g/||g||) (x_1/||x_1||)^T, not Q."""
    from oracle.hd import HaarOracle
    n = 12
    x1 = torch.tensor(np.random.default_rng(2).standard_normal(n), dtype=F64, requires_grad=True)
    ora = HaarOracle(n, 1, 3)
    y = ora.apply(x1)
    J = torch.stack([torch.autograd.grad(y[i], x1, retain_graph=True)[0] for i in range(n)])
    g = ora.g[0]
    want = torch.outer(g / g.norm(), x1.detach() / x1.detach().norm())
    assert torch.allclose(J, want, atol=1e-13)


def _dense_q(ens, n, rng):
    """Direct simulation: Ginibre iid N(0, 1/n); Haar by QR of a Gaussian with the signs of
    diag(R) moved into Q (Mezzadri's fix), which makes Q Haar distributed."""
    G = rng.standard_normal((n, n))
    if ens == "ginibre":
        return torch.tensor(G / np.sqrt(n), dtype=F64)
    q, r = np.linalg.qr(G)
    return torch.tensor(q * np.sign(np.diag(r)), dtype=F64)


@pytest.mark.parametrize("ens", ["haar", "ginibre"])
def test_mean_pathwise_gradient_matches_dense_simulation(ens):
    """The sampler's output has the law of the direct simulation for every parameter value
    (Theorems 1 and 2), so with smooth dynamics the mean of the pathwise derivative (draws held
    fixed) equals the derivative of the mean, which the dense simulation estimates too.  Per
    sample the two derivatives differ (the Haar step-1 Jacobian is rank one); their means over
    independent trials agree within 4.5 standard errors, component by component."""
    n, T, trials = 16, 4, 1200
    sched = [False, True, False, True]
    sigma = 1.0 if ens == "haar" else n ** -0.5
    rng = np.random.default_rng(31)
    x1 = torch.tensor(rng.standard_normal(n), dtype=F64)
    c = torch.tensor(rng.standard_normal(n), dtype=F64)
    theta0 = torch.tensor([0.9, 1.3, 0.7, 1.1], dtype=F64)

    def grads(apply):
        th = theta0.clone().requires_grad_(True)
        b = torch.tensor(0.4, dtype=F64, requires_grad=True)
        x, xprev = x1, None
        for t in range(1, T + 1):
            x, xprev = f_theta(t, apply(x, sched[t - 1]), x, xprev, th, b), x
        gt, gb = torch.autograd.grad(torch.dot(c, x), (th, b))
        return torch.cat([gt, gb.reshape(1)]).numpy()

    hd = np.array([grads(lambda x, tr, o=make_oracle(ens, n, n, T, 7, trial=i, sigma=sigma):
                         o.apply(x, tr)) for i in range(trials)])
    dense = []
    for _ in range(trials):
        Q = _dense_q(ens, n, rng)
        dense.append(grads(lambda x, tr, Q=Q: Q.T @ x if tr else Q @ x))
    dense = np.array(dense)
    se = np.sqrt(hd.var(axis=0, ddof=1) / trials + dense.var(axis=0, ddof=1) / trials)
    gap = np.abs(hd.mean(axis=0) - dense.mean(axis=0))
    assert (gap <= 4.5 * se).all(), (gap / se)
    # the means are informative (not both near zero within their noise)
    assert (np.abs(dense.mean(axis=0)) > 2.0 * se).sum() >= 2, dense.mean(axis=0) / se
