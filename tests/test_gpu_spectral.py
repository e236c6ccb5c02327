"""The spectral method of Section 2.2 on the GPU (the caller's dynamics around hd_apply):
measurements y = tanh(|Q^T [xi; 0]|) and power iterations x <- D x / ||D x|| with
D x = (1/m) [I 0] Q (y o Q^T [x; 0]), Q ~ Haar(m), m = 2n.  Every iterate equals the
oracle's (FP64 1e-10, FP32 1e-4; 17 products, Q^T and Q alternating)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def power_iteration(apply, xi, x0, n, m, K):
    """The same steps as oracle.spectral.power_iteration; apply(v, transpose) is one product."""
    z = torch.zeros(m - n, dtype=xi.dtype, device=xi.device)
    y = torch.tanh(torch.abs(apply(torch.cat([xi, z]), True)))
    x = x0 / torch.linalg.vector_norm(x0)
    xs = []
    for _ in range(K):
        u = apply(torch.cat([x, z]), True)
        v = apply(y * u, False)[:n] / m
        x = v / torch.linalg.vector_norm(v)
        xs.append(x)
    return y, xs


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_spectral_power_iteration_matches_oracle(dtype, tol):
    from oracle.hd import HaarOracle
    from oracle.spectral import power_iteration as oracle_power
    from paper_2101_07464_gb300 import HD
    n, K, seed = 3001, 8, 12
    m = 2 * n
    tdt = torch.float64 if dtype == "f64" else torch.float32
    xi, x0 = synth.x1(n, seed), synth.x1(n, seed + 1)
    if dtype == "f32":
        xi, x0 = (v.astype(np.float32).astype(np.float64) for v in (xi, x0))
    st = HD("haar", m, m, 1 + 2 * K, seed, dtype)
    yg, xg = power_iteration(st.apply, torch.tensor(xi, dtype=tdt, device="cuda"),
                             torch.tensor(x0, dtype=tdt, device="cuda"), n, m, K)
    st.close()
    yo, xo = oracle_power(HaarOracle(m, 1 + 2 * K, seed), xi, n, m, K, x0)
    assert torch.linalg.vector_norm(yg.double().cpu() - yo) <= tol * torch.linalg.vector_norm(yo)
    for k in range(K):
        err = torch.linalg.vector_norm(xg[k].double().cpu() - xo[k]).item()
        assert err <= tol, (k, err)
