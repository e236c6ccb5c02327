"""Differentiable ISTA on Householder Dice (the 64-trial ISTA workload's dynamics, Section 2.1
of the paper with A = Q square Gaussian, entries N(0, 1/n)):

    y = Q beta* + w;  x^0 = 0;  x^{k+1} = eta(x^k + tau Q^T (y - Q x^k); theta_k),

eta the soft threshold, beta* ~ 0.2 delta_0 + 0.8 N(0, 2^2), w ~ N(0, 0.1^2).  As products:
t = 1 is Q beta*, then Q x^k and Q^T r^k alternate (2K + 1 products for K iterations).  The
loss (1/n) ||x^K - beta*||^2 is differentiated with respect to theta_1..theta_K and tau
through the library's reverse mode (autograd.trajectory), the draws held fixed:

* FP64 gradients equal the oracle's torch float64 autograd (relative 1e-9);
* they equal central finite differences of the GPU FP64 forward (h = 1e-6: the soft
  threshold's kinks make wider differences cross them);
* FP32 gradients agree with FP64 ones to 1e-3 at n = 20000.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


from dyn_util import ista_f, ista_schedule as schedule   # noqa: E402


def inputs(n, seed, dtype):
    beta = synth.bernoulli_gauss(n, seed, p_nonzero=0.8, scale=2.0, dtype=dtype)
    w = synth.noise(n, seed, sigma=0.1, dtype=dtype)
    return beta, w


def gpu_loss_grad(n, K, seed, dtype, theta, tau, grad=True):
    from paper_2101_07464_gb300 import HD
    from paper_2101_07464_gb300.autograd import trajectory
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    beta, w = inputs(n, seed, npdt)
    bt = torch.tensor(beta, dtype=tdt, device="cuda")
    wt = torch.tensor(w, dtype=tdt, device="cuda")
    st = HD("ginibre", n, n, 2 * K + 1, seed, dtype, sigma=n ** -0.5)
    th = torch.tensor(theta, dtype=tdt, device="cuda", requires_grad=grad)
    ta = torch.tensor(tau, dtype=tdt, device="cuda", requires_grad=grad)
    xK = trajectory(st, bt, schedule(K), ista_f(wt), (th, ta))
    L = torch.sum((xK - bt) ** 2) / n
    out = [L.item()]
    if grad:
        L.backward()
        out += [th.grad.double().cpu().numpy(), ta.grad.item()]
    st.close()
    return out


def test_ista_fp64_gradients_match_oracle_autograd():
    from oracle.adjoint import trajectory as oracle_trajectory
    n, K, seed = 1000, 10, 3
    theta, tau = np.full(K, 0.6), 0.3
    Lg, gth, gta = gpu_loss_grad(n, K, seed, "f64", theta, tau)
    beta, w = inputs(n, seed, np.float64)
    bt, wt = torch.tensor(beta), torch.tensor(w)
    th = torch.tensor(theta, requires_grad=True)
    ta = torch.tensor(tau, dtype=torch.float64, requires_grad=True)
    xK = oracle_trajectory("ginibre", n, n, 2 * K + 1, seed, schedule(K), ista_f(wt), bt, (th, ta),
                           sigma=n ** -0.5)
    Lo = torch.sum((xK - bt) ** 2) / n
    Lo.backward()
    assert abs(Lg - Lo.item()) <= 1e-11 * abs(Lo.item())
    assert np.linalg.norm(gth - th.grad.numpy()) <= 1e-9 * np.linalg.norm(th.grad.numpy())
    assert abs(gta - ta.grad.item()) <= 1e-9 * abs(ta.grad.item())


def test_ista_fp64_gradients_match_finite_differences():
    """The loss is piecewise smooth: an iterate component within h of its threshold puts a
    kink inside the difference.  h = 1e-4 met one here (0.9 % off for theta_1), so the
    differences use h = 1e-6, which FP64 still resolves to about 1e-9."""
    n, K, seed = 2000, 8, 5
    theta, tau, h = np.full(K, 0.6), 0.3, 1e-6
    _, gth, gta = gpu_loss_grad(n, K, seed, "f64", theta, tau)
    for j in (0, K // 2, K - 1):
        e = np.zeros(K)
        e[j] = h
        fd = (gpu_loss_grad(n, K, seed, "f64", theta + e, tau, grad=False)[0] -
              gpu_loss_grad(n, K, seed, "f64", theta - e, tau, grad=False)[0]) / (2 * h)
        assert abs(fd - gth[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, gth[j])
    fd = (gpu_loss_grad(n, K, seed, "f64", theta, tau + h, grad=False)[0] -
          gpu_loss_grad(n, K, seed, "f64", theta, tau - h, grad=False)[0]) / (2 * h)
    assert abs(fd - gta) <= 1e-6 * max(1.0, abs(fd)), (fd, gta)


def test_ista_fp32_gradients_agree_with_fp64():
    n, K, seed = 20_000, 10, 7
    theta, tau = np.full(K, 0.6), 0.3
    L64, g64, t64 = gpu_loss_grad(n, K, seed, "f64", theta, tau)
    L32, g32, t32 = gpu_loss_grad(n, K, seed, "f32", theta, tau)
    assert abs(L32 - L64) <= 1e-4 * abs(L64)
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64)
    assert abs(t32 - t64) <= 1e-3 * abs(t64)
