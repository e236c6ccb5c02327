"""Batched ISTA for the lasso as a built-in dynamics of hd_run (HD_DYN_ISTA; Section 2.1):
every trial's products and ISTA updates against the oracle's ISTA, teacher-forced, element by
element; and the paper's Fig. 1a comparison on the GPU: the mean MSE curve of HD over many
independent trials agrees with direct simulation on dense Gaussian matrices.

Workload of the Fig. 1 caption: Gin(m, n), m = n/2, entries N(0, 1/m), beta* ~ 0.2 delta_0 +
0.8 N(0, 2^2), w ~ N(0, 0.1^2), tau = 0.3, threshold lambda tau = 0.6.
"""
import numpy as np
import pytest
from scipy import stats

import synth
from gpu_util import TOL, elem_err, f32_cast
from oracle.dynamics import ista_trace

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALT = lambda t: t % 2 == 0
TAU, THETA = 0.3, 0.6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lasso_inputs(n, m, seed, i):
    return (synth.bernoulli_gauss(n, seed, trial=i, p_nonzero=0.8, scale=2.0),
            synth.noise(m, seed, trial=i, sigma=0.1))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_ista_teacher_forced_elementwise(dtype):
    import paper_2101_07464_gb300 as hd
    from oracle.hd import GinibreOracle
    ns = [1000, 2003, 30_011, 777]
    ms = [n // 2 for n in ns]
    T, seed = 24, 31
    tdt = torch.float64 if dtype == "f64" else torch.float32
    cast = f32_cast if dtype == "f32" else None
    traces = []
    for i, (n, m) in enumerate(zip(ns, ms)):
        beta, w = lasso_inputs(n, m, seed, i)
        if cast is not None:
            beta, w = cast(beta), cast(w)
        ora = GinibreOracle(m, n, T, seed, trial=i, sigma=m ** -0.5)
        traces.append((beta, w, ista_trace(ora, beta, w, T, THETA, TAU, cast=cast)))
    b = hd.HDBatch("ginibre", ms, ns, T, seed, dtype)
    b.set_trial_sigmas([m ** -0.5 for m in ms])
    off_n, off_m = b.off_n, b.off_m
    L = int(max(off_n[-1], off_m[-1]))
    given = torch.zeros((T, L), dtype=tdt, device="cuda")
    for t in range(1, T):
        row = np.concatenate([tr[2]["used"][t - 1] for tr in traces])
        given[t - 1, :row.shape[0]] = torch.tensor(row, dtype=tdt)
    yrec = torch.zeros((T, L), dtype=tdt, device="cuda")
    xrec = torch.zeros((T, L), dtype=tdt, device="cuda")
    beta = torch.tensor(np.concatenate([tr[0] for tr in traces]), dtype=tdt, device="cuda")
    w = torch.tensor(np.concatenate([tr[1] for tr in traces]), dtype=tdt, device="cuda")
    out = torch.empty(int(off_n[-1]), dtype=tdt, device="cuda")
    spec = hd.make_run_spec([ALT(t) for t in range(1, T + 1)], "ista", THETA, use_graph=True, aux=w,
                            y_record=yrec, x_record=xrec, x_given=given, b=TAU)
    hd.hd_run(b.h, spec, beta, out)
    torch.cuda.synchronize()
    b.close()
    yrec, xrec = yrec.double().cpu().numpy(), xrec.double().cpu().numpy()
    tol = TOL[dtype]
    for t in range(1, T + 1):
        off = off_n if t % 2 == 0 else off_m
        for i, tr in enumerate(traces):
            lo, hi = int(off[i]), int(off[i + 1])
            assert elem_err(yrec[t - 1, lo:hi], tr[2]["products"][t - 1], t) <= tol, (t, i)
            assert elem_err(xrec[t - 1, lo:hi], tr[2]["updates"][t - 1], t) <= tol, (t, i)


def gpu_mse_curve(n, K, trials, seed, dtype="f32"):
    """Mean MSE (1/n) ||x^k - beta*||^2 per iteration k over `trials` independent trials of HD
    ISTA in one batched state (one CUDA graph), from the recorded x^k."""
    import paper_2101_07464_gb300 as hd
    m = n // 2
    T = 2 * K
    tdt = torch.float64 if dtype == "f64" else torch.float32
    b = hd.HDBatch("ginibre", [m] * trials, [n] * trials, T, seed, dtype)
    b.set_trial_sigmas([m ** -0.5] * trials)
    beta = np.concatenate([lasso_inputs(n, m, seed, i)[0] for i in range(trials)])
    w = np.concatenate([lasso_inputs(n, m, seed, i)[1] for i in range(trials)])
    bt = torch.tensor(beta, dtype=tdt, device="cuda")
    wt = torch.tensor(w, dtype=tdt, device="cuda")
    xrec = torch.zeros((T, n * trials), dtype=tdt, device="cuda")
    out = torch.empty(n * trials, dtype=tdt, device="cuda")
    spec = hd.make_run_spec([ALT(t) for t in range(1, T + 1)], "ista", THETA, use_graph=True, aux=wt,
                            x_record=xrec, b=TAU)
    hd.hd_run(b.h, spec, bt, out)
    torch.cuda.synchronize()
    b.close()
    xs = xrec[1::2].double().reshape(K, trials, n)                # x^1 .. x^K
    mse = ((xs - bt.double().reshape(1, trials, n)) ** 2).mean(dim=2)   # K x trials
    return mse.t().cpu().numpy()


def direct_curve(n, K, rng):
    """ISTA on a dense Gin(n/2, n) matrix with entries N(0, 1/m) (the direct approach)."""
    from oracle.direct import ginibre
    m = n // 2
    beta = (rng.random(n) < 0.8) * 2.0 * rng.standard_normal(n)
    w = 0.1 * rng.standard_normal(m)
    A = ginibre(rng, m, n, m ** -0.5)
    y = A @ beta + w
    x, mse = np.zeros(n), []
    for _ in range(K):
        v = x + TAU * (A.T @ (y - A @ x))
        x = np.sign(v) * np.maximum(np.abs(v) - THETA, 0.0)
        mse.append(float(np.sum((x - beta) ** 2) / n))
    return mse


def test_fig1a_mse_curve_matches_direct_simulation():
    """Fig. 1a at n = 400: 4000 HD trials on the GPU against 1000 direct simulations on dense
    matrices (oracle/direct.py); per iteration the mean MSEs agree within 4 combined standard
    errors, and the final MSEs pass a two-sample KS test."""
    n, K = 400, 25
    hd_mse = gpu_mse_curve(n, K, 4000, 5)
    rng = np.random.default_rng(77)
    dr = np.array([direct_curve(n, K, rng) for _ in range(1000)])
    se = np.sqrt(hd_mse.var(axis=0, ddof=1) / hd_mse.shape[0] + dr.var(axis=0, ddof=1) / dr.shape[0])
    gap = np.abs(hd_mse.mean(axis=0) - dr.mean(axis=0))
    assert (gap <= 4.0 * se).all(), gap / se
    assert stats.ks_2samp(hd_mse[:, -1], dr[:, -1]).pvalue > 1e-3
    # the iterations move away from x^0 = 0, whose MSE is E beta*^2 = 0.8 * 4
    assert hd_mse.mean(axis=0)[-1] < 0.9 * 3.2
