"""Reverse mode on the GPU (hd_adjoint_* through paper_2101_07464_gb300.autograd.trajectory).

* FP64 gradients of a loss of x_{T+1} with respect to x_1 and to the parameters of f_t equal
  the oracle's torch float64 autograd on the same seed (relative 1e-9): Haar and Ginibre, Q /
  Q^T alternating, all Q, mixed schedules, rectangular both ways, several CTAs.
* They equal central finite differences of the GPU FP64 forward (relative 1e-6), with the
  step h = 1e-4 on smooth dynamics and 1e-5 elsewhere.
* The FP32 reverse mode agrees with the oracle's FP64 autograd and with the FP64 reverse mode
  to 1e-4 (relative).
* Segment checkpointing (recompute with hd_probe) gives the recorded result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.adjoint import trajectory as oracle_trajectory   # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def f_theta(t, y, x, xprev, theta, beta):
    v = torch.tanh(theta[t - 1] * y)
    return v if xprev is None else v + beta * xprev


def f_square(t, y, x, xprev, theta, beta):
    return torch.tanh(theta[t - 1] * y) + beta * x


ALT = lambda T: [t % 2 == 0 for t in range(1, T + 1)]
ALLQ = lambda T: [False] * T
MIX = lambda T: [t in (2, 3, 6, 9) for t in range(1, T + 1)]

CASES = [
    ("haar", 300, 300, 12, ALT, f_theta),
    ("haar", 257, 257, 10, ALLQ, f_square),
    ("haar", 5003, 5003, 14, MIX, f_square),
    ("ginibre", 200, 330, 12, ALT, f_theta),
    ("ginibre", 331, 190, 11, ALT, f_theta),
    ("ginibre", 250, 250, 9, ALLQ, f_square),
    ("ginibre", 4001, 4001, 12, MIX, f_square),
]


def gpu_grads(ens, m, n, T, sched, f, x1, theta, beta, c, dtype, checkpoint=None, seed=11):
    from paper_2101_07464_gb300 import HD
    from paper_2101_07464_gb300.autograd import trajectory
    tdt = torch.float64 if dtype == "f64" else torch.float32
    sigma = 1.0 if ens == "haar" else m ** -0.5
    hd = HD(ens, m, n, T, seed, dtype, sigma=sigma)
    xt = torch.tensor(x1, dtype=tdt, device="cuda", requires_grad=True)
    th = torch.tensor(theta, dtype=tdt, device="cuda", requires_grad=True)
    be = torch.tensor(beta, dtype=tdt, device="cuda", requires_grad=True)
    out = trajectory(hd, xt, sched, f, (th, be), checkpoint=checkpoint)
    L = torch.dot(torch.tensor(c, dtype=tdt, device="cuda"), out)
    L.backward()
    res = (L.item(), xt.grad.double().cpu().numpy(), th.grad.double().cpu().numpy(), be.grad.item())
    hd.close()
    return res


def oracle_grads(ens, m, n, T, sched, f, x1, theta, beta, c, seed=11):
    F64 = torch.float64
    sigma = 1.0 if ens == "haar" else m ** -0.5
    xt = torch.tensor(x1, dtype=F64, requires_grad=True)
    th = torch.tensor(theta, dtype=F64, requires_grad=True)
    be = torch.tensor(beta, dtype=F64, requires_grad=True)
    out = oracle_trajectory(ens, m, n, T, seed, sched, f, xt, (th, be), sigma=sigma)
    L = torch.dot(torch.tensor(c, dtype=F64), out)
    L.backward()
    return L.item(), xt.grad.numpy(), th.grad.numpy(), be.grad.item()


def rel(a, b):
    a, b = np.atleast_1d(a), np.atleast_1d(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(ens, m, n, T, schedf, seed=3):
    sched = schedf(T)
    rng = np.random.default_rng(seed)
    x1 = rng.standard_normal(m if sched[0] else n)
    theta = 0.6 + 0.4 * rng.random(T)
    # x_{T+1} lives where y_T does
    c = rng.standard_normal(n if sched[-1] else m)
    return sched, x1, theta, 0.3, c


@pytest.mark.parametrize("ens,m,n,T,schedf,f", CASES)
def test_fp64_adjoint_matches_oracle_autograd(ens, m, n, T, schedf, f):
    sched, x1, theta, beta, c = _case(ens, m, n, T, schedf)
    Lg, gx, gt, gb = gpu_grads(ens, m, n, T, sched, f, x1, theta, beta, c, "f64")
    Lo, ox, ot, ob = oracle_grads(ens, m, n, T, sched, f, x1, theta, beta, c)
    assert abs(Lg - Lo) <= 1e-11 * max(1.0, abs(Lo))
    assert rel(gx, ox) <= 1e-9, rel(gx, ox)
    assert rel(gt, ot) <= 1e-9, rel(gt, ot)
    assert rel(gb, ob) <= 1e-9, (gb, ob)


def _f32(v):
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("ens,m,n,T,schedf,f", CASES + [
    ("haar", 100_003, 100_003, 16, ALT, f_theta),
    ("ginibre", 40_000, 70_001, 12, ALT, f_theta)])
def test_fp32_adjoint_matches_oracle_autograd(ens, m, n, T, schedf, f):
    """The FP32 reverse mode (FP32 stacks and passes, FP64 sums and coefficients) against the
    oracle's FP64 autograd on the same FP32-representable inputs, relative 1e-4."""
    sched, x1, theta, beta, c = _case(ens, m, n, T, schedf, seed=5)
    x1, theta, c = _f32(x1), _f32(theta), _f32(c)
    beta = float(np.float32(beta))
    Lg, gx, gt, gb = gpu_grads(ens, m, n, T, sched, f, x1, theta, beta, c, "f32")
    Lo, ox, ot, ob = oracle_grads(ens, m, n, T, sched, f, x1, theta, beta, c)
    assert abs(Lg - Lo) <= 1e-4 * max(1.0, abs(Lo)), (Lg, Lo)
    assert rel(gx, ox) <= 1e-4, rel(gx, ox)
    assert rel(gt, ot) <= 1e-4, rel(gt, ot)
    assert rel(gb, ob) <= 1e-4, (gb, ob)


@pytest.mark.parametrize("ens,m,n,T,schedf,f", [CASES[0], CASES[3], CASES[6]])
def test_fp64_adjoint_matches_finite_differences(ens, m, n, T, schedf, f):
    from paper_2101_07464_gb300 import HD
    sched, x1, theta, beta, c = _case(ens, m, n, T, schedf, seed=8)
    _, gx, gt, gb = gpu_grads(ens, m, n, T, sched, f, x1, theta, beta, c, "f64")
    sigma = 1.0 if ens == "haar" else m ** -0.5
    hd = HD(ens, m, n, T, 11, "f64", sigma=sigma)
    cd = torch.tensor(c, dtype=torch.float64, device="cuda")

    def L(x1_, th_, b_):
        hd.reset()
        x = torch.tensor(x1_, dtype=torch.float64, device="cuda")
        th = torch.tensor(th_, dtype=torch.float64, device="cuda")
        xp = None
        for t in range(1, T + 1):
            y = hd.apply(x, sched[t - 1])
            x, xp = f(t, y, x, xp, th, b_), x
        return torch.dot(cd, x).item()

    h = 1e-5
    rng = np.random.default_rng(1)
    v = rng.standard_normal(x1.size)
    fd = (L(x1 + h * v, theta, beta) - L(x1 - h * v, theta, beta)) / (2 * h)
    assert abs(fd - gx @ v) <= 1e-6 * max(1.0, abs(fd)), (fd, gx @ v)
    e = np.zeros(T)
    e[T // 2] = 1.0
    fd = (L(x1, theta + h * e, beta) - L(x1, theta - h * e, beta)) / (2 * h)
    assert abs(fd - gt[T // 2]) <= 1e-6 * max(1.0, abs(fd)), (fd, gt[T // 2])
    hd.close()


@pytest.mark.parametrize("ens,m,n,T,schedf,f", [CASES[0], CASES[3], CASES[5]])
def test_fp64_adjoint_matches_central_differences_at_h_1e4(ens, m, n, T, schedf, f):
    """Central differences with the step h = 1e-4 on these smooth dynamics (tanh, no kinks):
    the truncation error is O(h^2), so directional derivatives agree to 1e-6 relative."""
    from paper_2101_07464_gb300 import HD
    sched, x1, theta, beta, c = _case(ens, m, n, T, schedf, seed=12)
    _, gx, gt, gb = gpu_grads(ens, m, n, T, sched, f, x1, theta, beta, c, "f64")
    sigma = 1.0 if ens == "haar" else m ** -0.5
    hd = HD(ens, m, n, T, 11, "f64", sigma=sigma)
    cd = torch.tensor(c, dtype=torch.float64, device="cuda")

    def L(x1_, th_, b_):
        hd.reset()
        x = torch.tensor(x1_, dtype=torch.float64, device="cuda")
        th = torch.tensor(th_, dtype=torch.float64, device="cuda")
        xp = None
        for t in range(1, T + 1):
            y = hd.apply(x, sched[t - 1])
            x, xp = f(t, y, x, xp, th, b_), x
        return torch.dot(cd, x).item()

    h = 1e-4
    v = np.random.default_rng(2).standard_normal(x1.size)
    v /= np.linalg.norm(v)
    fd = (L(x1 + h * v, theta, beta) - L(x1 - h * v, theta, beta)) / (2 * h)
    assert abs(fd - gx @ v) <= 1e-6 * max(1.0, abs(fd)), (fd, gx @ v)
    e = np.random.default_rng(3).standard_normal(T)
    e /= np.linalg.norm(e)
    fd = (L(x1, theta + h * e, beta) - L(x1, theta - h * e, beta)) / (2 * h)
    assert abs(fd - gt @ e) <= 1e-6 * max(1.0, abs(fd)), (fd, gt @ e)
    fd = (L(x1, theta, beta + h) - L(x1, theta, beta - h)) / (2 * h)
    assert abs(fd - gb) <= 1e-6 * max(1.0, abs(fd)), (fd, gb)
    hd.close()


@pytest.mark.parametrize("ens,m,n,T,schedf,f", [
    ("haar", 100_003, 100_003, 16, ALT, f_theta),    # rows not a multiple of 4: scalar passes
    ("haar", 100_000, 100_000, 16, ALT, f_theta),    # 16-byte vector passes
    ("ginibre", 40_000, 70_001, 12, ALT, f_theta)])
def test_fp32_adjoint_matches_fp64(ens, m, n, T, schedf, f):
    sched, x1, theta, beta, c = _case(ens, m, n, T, schedf, seed=4)
    _, gx64, gt64, gb64 = gpu_grads(ens, m, n, T, sched, f, x1, theta, beta, c, "f64")
    _, gx32, gt32, gb32 = gpu_grads(ens, m, n, T, sched, f, x1, theta, beta, c, "f32")
    assert rel(gx32, gx64) <= 1e-4, rel(gx32, gx64)
    assert rel(gt32, gt64) <= 1e-4, rel(gt32, gt64)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_checkpointed_matches_recorded(dtype):
    ens, m, n, T = "haar", 20_011, 20_011, 20
    sched, x1, theta, beta, c = _case(ens, m, n, T, ALT, seed=6)
    _, gx, gt, gb = gpu_grads(ens, m, n, T, sched, f_theta, x1, theta, beta, c, dtype)
    _, cx, ct, cb = gpu_grads(ens, m, n, T, sched, f_theta, x1, theta, beta, c, dtype, checkpoint=6)
    tol = 1e-10 if dtype == "f64" else 1e-4
    assert rel(cx, gx) <= tol, rel(cx, gx)
    assert rel(ct, gt) <= tol, rel(ct, gt)


def test_reverse_mode_state_rules():
    from paper_2101_07464_gb300 import HD, HDError, hd_adjoint_position
    hd = HD("haar", 64, 64, 4, 1, "f64")
    x = torch.randn(64, dtype=torch.float64, device="cuda")
    hd.apply(x)
    with pytest.raises(HDError) as ei:   # steps already taken
        hd.adjoint_enable()
    assert ei.value.code == 7
    hd.reset()
    hd.adjoint_enable()
    y1 = hd.apply(x)
    y2 = hd.apply(torch.tanh(y1), True)
    assert hd_adjoint_position(hd.h) == 2
    hd.adjoint_step(torch.ones_like(y2), True)
    with pytest.raises(HDError) as ei:   # no forward steps once the reverse pass started
        hd.apply(x)
    assert ei.value.code == 7
    hd.adjoint_step(torch.ones_like(y1), False)
    with pytest.raises(HDError) as ei:   # everything reversed
        hd.adjoint_step(torch.ones_like(y1), False)
    assert ei.value.code == 7
    hd.close()
