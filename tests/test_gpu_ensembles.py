"""GOE and U Sigma V products on the GPU (hd_goe_apply, hd_usv_apply) against the oracle's
compositions (paper, section "Other Random Matrix Ensembles"):

* teacher-forced sequences of queries, FP64 to 1e-12 and FP32 to 1e-5 per query;
* GOE: the revealed block is symmetric; batched square Ginibre states give each trial's GOE;
* U Sigma V (eq. inv): at small sizes the reconstructed matrix has singular values s;
* argument errors.
"""
import math

import numpy as np
import pytest

import synth
from gpu_util import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_goe_teacher_forced(dtype):
    from oracle.ensembles import goe_apply, make_goe
    from paper_2101_07464_gb300 import HD
    n, q, seed = 5003, 8, 21
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ora = make_goe(n, 2 * q, seed, sigma=n ** -0.5)
    gpu = HD("ginibre", n, n, 2 * q, seed, dtype, sigma=n ** -0.5)
    x = synth.x1(n, seed)
    errs = []
    for _ in range(q):
        if dtype == "f32":
            x = x.astype(np.float32).astype(np.float64)
        yo = goe_apply(ora, x).numpy()
        yg = gpu.goe(torch.tensor(x, dtype=tdt, device="cuda")).double().cpu().numpy()
        errs.append(np.linalg.norm(yg - yo) / np.linalg.norm(yo))
        x = np.tanh(yo)
    gpu.close()
    assert max(errs) <= TOL[dtype], errs


def test_goe_symmetric_and_batched():
    import paper_2101_07464_gb300 as hd
    from oracle.ensembles import goe_apply, make_goe
    n, q = 40, 10
    st = hd.HD("ginibre", n, n, 2 * q, 3, "f64")
    cols = []
    for j in range(q):
        ej = torch.zeros(n, dtype=torch.float64, device="cuda")
        ej[j] = 1.0
        cols.append(st.goe(ej).cpu().numpy())
    W = np.stack(cols, axis=1)[:q, :]
    assert np.abs(W - W.T).max() <= 1e-13 * np.abs(W).max()
    st.close()
    # batched: each trial's GOE equals the oracle's for that trial (Philox trial word i)
    ns = [300, 1001, 64]
    b = hd.HDBatch("ginibre", ns, ns, 4, 9, "f64")
    xs = [synth.x1(nn, 9, trial=i) for i, nn in enumerate(ns)]
    x = torch.tensor(np.concatenate(xs), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    hd.hd_goe_apply(b.h, x, y)
    yc = y.cpu().numpy()
    for i, nn in enumerate(ns):
        yo = goe_apply(make_goe(nn, 4, 9, trial=i), xs[i]).numpy()
        yi = yc[b.off_n[i]:b.off_n[i + 1]]
        assert np.linalg.norm(yi - yo) <= 1e-12 * np.linalg.norm(yo), i
    b.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("m,n", [(3001, 5003), (4099, 2003)])
def test_usv_teacher_forced(dtype, m, n):
    from oracle.ensembles import make_usv, usv_apply
    from paper_2101_07464_gb300 import USV
    q = 10
    rng = np.random.default_rng(m + n)
    s = rng.uniform(0.2, 2.0, min(m, n))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    U, V = make_usv(m, n, q, 31, 32)
    gpu = USV(m, n, q, 31, 32, s, dtype)
    errs = []
    for t in range(q):
        tr = t % 3 == 1
        x = synth.x1(m if tr else n, 40 + t)
        if dtype == "f32":
            x = x.astype(np.float32).astype(np.float64)
        yo = usv_apply(U, V, s, x, transpose=tr).numpy()
        yg = gpu.apply(torch.tensor(x, dtype=tdt, device="cuda"), tr).double().cpu().numpy()
        errs.append(np.linalg.norm(yg - yo) / np.linalg.norm(yo))
    gpu.close()
    assert max(errs) <= TOL[dtype], errs


def test_usv_singular_values_and_errors():
    import paper_2101_07464_gb300 as hd
    m = n = 8
    s = np.array([3.0, 2.5, 2.0, 1.5, 1.0, 0.8, 0.5, 0.25])
    g = hd.USV(m, n, n, 5, 6, s, "f64")
    cols = []
    for j in range(n):
        ej = torch.zeros(n, dtype=torch.float64, device="cuda")
        ej[j] = 1.0
        cols.append(g.apply(ej).cpu().numpy())
    sv = np.linalg.svd(np.stack(cols, axis=1), compute_uv=False)
    np.testing.assert_allclose(np.sort(sv)[::-1], s, rtol=1e-12)
    g.close()
    haar = hd.HD("haar", 16, 16, 4, 1, "f64")
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(hd.HDError) as ei:   # GOE needs a Ginibre state
        hd.hd_goe_apply(haar.h, x, y)
    assert ei.value.code == 1
    rect = hd.HD("ginibre", 12, 16, 4, 1, "f64")
    with pytest.raises(hd.HDError) as ei:   # and a square one
        hd.hd_goe_apply(rect.h, x, y)
    assert ei.value.code == 2
    sd = torch.ones(16, dtype=torch.float64, device="cuda")
    with pytest.raises(hd.HDError) as ei:   # U Sigma V needs two Haar states
        hd.hd_usv_apply(haar.h, rect.h, sd, x, 0, y)
    assert ei.value.code == 1
    haar.close()
    rect.close()
