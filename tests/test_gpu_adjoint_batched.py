"""Batched reverse mode: a batched state whose trials share their dimensions reverses every
trial in one set of launches per step (packed vectors, grid z = trial).

* FP64: the gradients of sum_i <c_i, x_{T+1,i}> with respect to the packed x_1 and the shared
  parameters equal those of independent single-trial states (same seed, trial word i) to
  1e-11, and the oracle's float64 autograd summed over the trials to 1e-9 (Haar and Ginibre,
  alternating, mixed and all-Q schedules, rectangular both ways, several CTAs per trial).
* FP32 against the oracle's autograd to 1e-4.
* ISTA (the differentiable ISTA workload's dynamics, the soft threshold of Section 2.1) on a
  batch: gradients in the thresholds and the step size against the oracle's autograd.
* Unequal trials are rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.adjoint import trajectory as oracle_trajectory   # noqa: E402

ALT = lambda T: [t % 2 == 0 for t in range(1, T + 1)]
ALLQ = lambda T: [False] * T
MIX = lambda T: [t in (2, 3, 6, 9) for t in range(1, T + 1)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def f_theta(t, y, x, xprev, theta, beta):
    v = torch.tanh(theta[t - 1] * y)
    return v if xprev is None else v + beta * xprev


def problem(ens, m, n, T, schedf, count, seed):
    sched = schedf(T)
    rng = np.random.default_rng(seed)
    din = m if sched[0] else n
    dout = n if sched[-1] else m
    x1 = [rng.standard_normal(din) for _ in range(count)]
    c = [rng.standard_normal(dout) for _ in range(count)]
    theta = 0.6 + 0.4 * rng.random(T)
    return sched, x1, c, theta, 0.3


def batched_grads(ens, m, n, T, sched, x1, c, theta, beta, dtype, seed=11):
    import paper_2101_07464_gb300 as hd
    from paper_2101_07464_gb300.autograd import trajectory
    tdt = torch.float64 if dtype == "f64" else torch.float32
    count = len(x1)
    sigma = 1.0 if ens == "haar" else m ** -0.5
    b = hd.HDBatch(ens, [m] * count, [n] * count, T, seed, dtype, sigma=sigma)
    xt = torch.tensor(np.concatenate(x1), dtype=tdt, device="cuda", requires_grad=True)
    th = torch.tensor(theta, dtype=tdt, device="cuda", requires_grad=True)
    be = torch.tensor(beta, dtype=tdt, device="cuda", requires_grad=True)
    out = trajectory(b, xt, sched, f_theta, (th, be))
    L = torch.dot(torch.tensor(np.concatenate(c), dtype=tdt, device="cuda"), out)
    L.backward()
    res = (L.item(), xt.grad.double().cpu().numpy(), th.grad.double().cpu().numpy(), be.grad.item())
    b.close()
    return res


def single_grads(ens, m, n, T, sched, x1, c, theta, beta, seed=11):
    from paper_2101_07464_gb300 import HD
    from paper_2101_07464_gb300.autograd import trajectory
    sigma = 1.0 if ens == "haar" else m ** -0.5
    Ls, gx, gt, gb = 0.0, [], np.zeros(len(theta)), 0.0
    for i in range(len(x1)):
        st = HD(ens, m, n, T, seed, "f64", sigma=sigma, trial=i)
        xt = torch.tensor(x1[i], dtype=torch.float64, device="cuda", requires_grad=True)
        th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
        be = torch.tensor(beta, dtype=torch.float64, device="cuda", requires_grad=True)
        out = trajectory(st, xt, sched, f_theta, (th, be))
        L = torch.dot(torch.tensor(c[i], dtype=torch.float64, device="cuda"), out)
        L.backward()
        Ls += L.item()
        gx.append(xt.grad.cpu().numpy())
        gt += th.grad.cpu().numpy()
        gb += be.grad.item()
        st.close()
    return Ls, np.concatenate(gx), gt, gb


def oracle_grads(ens, m, n, T, sched, x1, c, theta, beta, seed=11):
    sigma = 1.0 if ens == "haar" else m ** -0.5
    Ls, gx, gt, gb = 0.0, [], np.zeros(len(theta)), 0.0
    for i in range(len(x1)):
        xt = torch.tensor(x1[i], dtype=torch.float64, requires_grad=True)
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        be = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        out = oracle_trajectory(ens, m, n, T, seed, sched, f_theta, xt, (th, be), trial=i, sigma=sigma)
        L = torch.dot(torch.tensor(c[i], dtype=torch.float64), out)
        L.backward()
        Ls += L.item()
        gx.append(xt.grad.numpy())
        gt += th.grad.numpy()
        gb += be.grad.item()
    return Ls, np.concatenate(gx), gt, gb


def rel(a, b):
    a, b = np.atleast_1d(a), np.atleast_1d(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [("haar", 5003, 5003, 12, ALT, 4), ("haar", 1000, 1000, 10, MIX, 3), ("ginibre", 2001, 3001, 10, ALT, 3),
         ("ginibre", 3001, 1999, 9, ALT, 2), ("ginibre", 1500, 1500, 8, ALLQ, 5), ("ginibre", 1500, 1500, 10, MIX, 3)]


@pytest.mark.parametrize("ens,m,n,T,schedf,count", CASES)
def test_batched_fp64_matches_single_trials_and_oracle(ens, m, n, T, schedf, count):
    sched, x1, c, theta, beta = problem(ens, m, n, T, schedf, count, 3)
    Lb, gxb, gtb, gbb = batched_grads(ens, m, n, T, sched, x1, c, theta, beta, "f64")
    Ls, gxs, gts, gbs = single_grads(ens, m, n, T, sched, x1, c, theta, beta)
    assert abs(Lb - Ls) <= 1e-11 * max(1.0, abs(Ls))
    assert rel(gxb, gxs) <= 1e-11 and rel(gtb, gts) <= 1e-11 and rel(gbb, gbs) <= 1e-11, \
        (rel(gxb, gxs), rel(gtb, gts), rel(gbb, gbs))
    Lo, gxo, gto, gbo = oracle_grads(ens, m, n, T, sched, x1, c, theta, beta)
    assert abs(Lb - Lo) <= 1e-10 * max(1.0, abs(Lo))
    assert rel(gxb, gxo) <= 1e-9 and rel(gtb, gto) <= 1e-9 and rel(gbb, gbo) <= 1e-9, \
        (rel(gxb, gxo), rel(gtb, gto), rel(gbb, gbo))


@pytest.mark.parametrize("ens,m,n,T,schedf,count", [CASES[0], CASES[2]])
def test_batched_fp32_matches_oracle(ens, m, n, T, schedf, count):
    f32 = lambda v: np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)
    sched, x1, c, theta, beta = problem(ens, m, n, T, schedf, count, 5)
    x1, c, theta = [f32(v) for v in x1], [f32(v) for v in c], f32(theta)
    beta = float(np.float32(beta))
    Lb, gxb, gtb, gbb = batched_grads(ens, m, n, T, sched, x1, c, theta, beta, "f32")
    Lo, gxo, gto, gbo = oracle_grads(ens, m, n, T, sched, x1, c, theta, beta)
    assert abs(Lb - Lo) <= 1e-4 * max(1.0, abs(Lo))
    assert rel(gxb, gxo) <= 1e-4 and rel(gtb, gto) <= 1e-4 and rel(gbb, gbo) <= 1e-4, \
        (rel(gxb, gxo), rel(gtb, gto), rel(gbb, gbo))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_ista_gradients_match_oracle(dtype):
    """The differentiable ISTA dynamics on a batch of 6 trials (Gin(n, n), entries N(0, 1/n)):
    the gradient of the mean over trials of (1/n) ||x^K - beta*||^2 in theta_1..theta_K and
    tau, against the oracle's autograd (FP64 1e-9, FP32 1e-4)."""
    import paper_2101_07464_gb300 as hd
    import synth
    from dyn_util import ista_f, ista_schedule
    from paper_2101_07464_gb300.autograd import trajectory
    n, K, count, seed = 3000, 8, 6, 9
    T = 2 * K + 1
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    betas = [synth.bernoulli_gauss(n, seed, trial=i, p_nonzero=0.8, scale=2.0, dtype=npdt).astype(np.float64)
             for i in range(count)]
    ws = [synth.noise(n, seed, trial=i, sigma=0.1, dtype=npdt).astype(np.float64) for i in range(count)]
    theta, tau = np.full(K, 0.6), 0.3
    if dtype == "f32":
        theta, tau = theta.astype(np.float32).astype(np.float64), float(np.float32(tau))
    b = hd.HDBatch("ginibre", [n] * count, [n] * count, T, seed, dtype, sigma=n ** -0.5)
    bt = torch.tensor(np.concatenate(betas), dtype=tdt, device="cuda")
    wt = torch.tensor(np.concatenate(ws), dtype=tdt, device="cuda")
    th = torch.tensor(theta, dtype=tdt, device="cuda", requires_grad=True)
    ta = torch.tensor(tau, dtype=tdt, device="cuda", requires_grad=True)
    xK = trajectory(b, bt, ista_schedule(K), ista_f(wt), (th, ta))
    L = torch.sum((xK - bt) ** 2) / (n * count)
    L.backward()
    gth, gta = th.grad.double().cpu().numpy(), ta.grad.item()
    b.close()
    Lo, gto, gtao = 0.0, np.zeros(K), 0.0
    for i in range(count):
        tho = torch.tensor(theta, requires_grad=True)
        tao = torch.tensor(tau, dtype=torch.float64, requires_grad=True)
        bo = torch.tensor(betas[i])
        xo = oracle_trajectory("ginibre", n, n, T, seed, ista_schedule(K), ista_f(torch.tensor(ws[i])), bo, (tho, tao),
                               trial=i, sigma=n ** -0.5)
        Li = torch.sum((xo - bo) ** 2) / (n * count)
        Li.backward()
        Lo += Li.item()
        gto += tho.grad.numpy()
        gtao += tao.grad.item()
    tol = 1e-9 if dtype == "f64" else 1e-4
    assert abs(L.item() - Lo) <= tol * abs(Lo)
    assert rel(gth, gto) <= tol, rel(gth, gto)
    assert abs(gta - gtao) <= tol * abs(gtao), (gta, gtao)


def test_unequal_batch_is_rejected():
    import paper_2101_07464_gb300 as hd
    b = hd.HDBatch("haar", [100, 101], [100, 101], 4, 1, "f64")
    with pytest.raises(hd.HDError) as ei:
        b.adjoint_enable()
    assert ei.value.code == hd.binding.HD_ERR_ARG
    b.close()
