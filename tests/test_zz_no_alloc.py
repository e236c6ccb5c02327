"""hd_first_product_noalloc: the allocation-free first product of a fresh matrix.

It must give what a new state gives at its first hd_apply (same seed, trial, sigma) within
the parity tolerances, on two calls in a row on one stream (the second call sees the
scratch the first one left), match the oracle's first product, allocate no device memory,
and reject sizes beyond its scratch with a clear error.  This file sorts last so that it also runs after
every other test has used the device.
"""
import pytest

import synth
from gpu_util import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _via_state(ens, dtype, m, n, transpose, seed, trial, sigma, x):
    from paper_2101_07464_gb300 import HD
    st = HD(ens, m, n, 1, seed, dtype, sigma=sigma, trial=trial)
    y = st.apply(x, transpose).clone()
    st.close()
    return y


def _rel(a, b):
    a, b = a.double(), b.double()
    den = b.norm().item()
    return (a - b).norm().item() / den if den > 0 else a.norm().item()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("ens,m,n,transpose", [
    ("haar", 100_003, 100_003, False), ("haar", 4097, 4097, True), ("haar", 1, 1, False),
    ("ginibre", 30_011, 70_001, False), ("ginibre", 30_011, 70_001, True),
    ("ginibre", 8191, 5, True)])
def test_two_calls_match_state_first_product(dtype, ens, m, n, transpose):
    import paper_2101_07464_gb300 as hd
    tdt = torch.float64 if dtype == "f64" else torch.float32
    nx, ny = (m, n) if transpose else (n, m)
    sigma = 1.0 if ens == "haar" else m ** -0.5
    xa = torch.tensor(synth.x1(nx, 21), dtype=tdt, device="cuda")
    xb = torch.tensor(synth.x1(nx, 22), dtype=tdt, device="cuda")
    ya = torch.empty(ny, dtype=tdt, device="cuda")
    yb = torch.empty(ny, dtype=tdt, device="cuda")
    # two calls in a row on one stream, different seeds / trials, no sync in between
    hd.hd_first_product_noalloc(ens, dtype, m, n, transpose, 1234, 3, sigma, xa, ya)
    hd.hd_first_product_noalloc(ens, dtype, m, n, transpose, 98765, 0, sigma, xb, yb)
    ra = _via_state(ens, dtype, m, n, transpose, 1234, 3, sigma, xa)
    rb = _via_state(ens, dtype, m, n, transpose, 98765, 0, sigma, xb)
    torch.cuda.synchronize()
    assert _rel(ya, ra) <= TOL[dtype]
    assert _rel(yb, rb) <= TOL[dtype]


def test_largest_size_and_zero_input():
    import paper_2101_07464_gb300 as hd
    n = 16_777_216
    x = torch.tensor(synth.x1(n, 5), dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    hd.hd_first_product_noalloc("haar", "f32", n, n, False, 7, 1, 1.0, x, y)
    ref = _via_state("haar", "f32", n, n, False, 7, 1, 1.0, x)
    torch.cuda.synchronize()
    assert _rel(y, ref) <= TOL["f32"]
    z = torch.zeros(1000, dtype=torch.float64, device="cuda")
    yz = torch.full((700,), 3.0, dtype=torch.float64, device="cuda")
    hd.hd_first_product_noalloc("ginibre", "f64", 700, 1000, False, 7, 1, 0.1, z, yz)
    torch.cuda.synchronize()
    assert torch.count_nonzero(yz).item() == 0


@pytest.mark.parametrize("ens,m,n,transpose", [("haar", 5003, 5003, False), ("ginibre", 3001, 7001, True)])
def test_matches_oracle_first_product(ens, m, n, transpose):
    """Directly against the oracle's first product (FP64, same seed and trial)."""
    import numpy as np
    import paper_2101_07464_gb300 as hd
    from oracle.hd import make_oracle
    nx, ny = (m, n) if transpose else (n, m)
    sigma = 1.0 if ens == "haar" else m ** -0.5
    x = synth.x1(nx, 31)
    y = torch.empty(ny, dtype=torch.float64, device="cuda")
    hd.hd_first_product_noalloc(ens, "f64", m, n, transpose, 77, 2, sigma, torch.tensor(x, device="cuda"), y)
    yo = make_oracle(ens, m, n, 1, 77, trial=2, sigma=sigma).apply(x, transpose).numpy()
    torch.cuda.synchronize()
    yg = y.cpu().numpy()
    assert np.abs(yg - yo).max() <= TOL["f64"] * np.abs(yo).max()
    assert np.linalg.norm(yg - yo) <= TOL["f64"] * np.linalg.norm(yo)


def _free_bytes():
    """Free device memory, read until two readings agree (other users of the device can move
    it between readings)."""
    last = None
    for _ in range(10):
        torch.cuda.synchronize()
        f, _ = torch.cuda.mem_get_info()
        if f == last:
            return f
        last = f
    return last


def test_allocates_no_device_memory():
    """Device memory only (host allocations are not measured here)."""
    import paper_2101_07464_gb300 as hd
    n = 1_000_003
    x = torch.tensor(synth.x1(n, 9), dtype=torch.float64, device="cuda")
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    hd.hd_first_product_noalloc("haar", "f64", n, n, False, 1, 0, 1.0, x, y)   # first call on the device
    torch.cuda.synchronize()
    alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    free0 = _free_bytes()
    for k in range(20):
        hd.hd_first_product_noalloc("haar", "f64", n, n, k % 2 == 1, k, k, 1.0, x, y)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0
    assert _free_bytes() == free0


def test_rejects_oversize_and_bad_arguments():
    from paper_2101_07464_gb300.binding import lib
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    big = 16_777_217
    rc = lib().hd_first_product_noalloc(1, 0, big, big, 0, 1, 0, 1.0, x.data_ptr(), x.data_ptr(), None)
    assert rc == 2
    msg = lib().hd_last_error().decode()
    assert "16777216" in msg and "exceeds" in msg
    rc = lib().hd_first_product_noalloc(1, 0, 8, 9, 0, 1, 0, 1.0, x.data_ptr(), x.data_ptr(), None)
    assert rc == 2   # Haar needs m == n
    rc = lib().hd_first_product_noalloc(0, 0, 8, 8, 0, 1, 0, float("nan"), x.data_ptr(), x.data_ptr(), None)
    assert rc == 1
    rc = lib().hd_first_product_noalloc(1, 0, 8, 8, 0, 1, 0, 1.0, None, x.data_ptr(), None)
    assert rc == 1
