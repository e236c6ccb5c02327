"""Complex Householder Dice on the GPU (hd_complex_*: Q ~ Haar on the unitary group, complex
Ginibre and GUE, the paper's section "Other Random Matrix Ensembles", eq. Householder_c)
against the complex oracle (oracle/complex_hd.py), teacher-forced: both sides get the same x_t, and per step the norm
error ||y_gpu - y_ora|| / ||y_ora|| and the element-wise error (pivot rows relative to the
norm, the others to the largest entry; gpu_util.elem_err) are at most 1e-12 (complex FP64)
or 1e-5 (complex FP32).  Sizes span one to many CTAs with ragged ends, T = n, every schedule
of Q and Q^H; unitarity ||y_t|| = ||x_t|| holds to 1e-13 (FP64) at every step.

The dynamics is the entrywise phase map x_{t+1} = y_t / |y_t|, the complex counterpart of the
sign dynamics.  Under Q / Q^H alternation it converges: the part of x_t that the revealed
reflectors do not already fix, alpha_t / ||x_t|| from the oracle, falls from 1 to 1e-4 within
about 20 steps at n = 1000.  Per-step parity is then asserted while that fraction stays above
the unit roundoff over the tolerance (gpu_util.COND_MIN, readings A13(i) and A18); later
steps are checked for unitarity only."""
import numpy as np
import pytest

from gpu_util import COND_MIN, TOL, elem_err
from oracle.complex_hd import ComplexHaarOracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALT = lambda t: t % 2 == 0
ALLQ = lambda t: False
MIXED = lambda t: t in (2, 3, 7, 8, 9, 14)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def crand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def to_dtype(v, dtype):
    v = np.asarray(v, dtype=np.complex128)
    return v.astype(np.complex64).astype(np.complex128) if dtype == "f32" else v


def next_input(y):
    """The entrywise phase of the output: x_{t+1} = y_t / |y_t| (0 where y_t is 0)."""
    a = np.abs(y)
    return np.where(a > 0, y / np.where(a > 0, a, 1.0), 0.0)


def teacher_forced(n, T, seed, dtype, sched, trial=0):
    from paper_2101_07464_gb300 import HDComplex
    ora = ComplexHaarOracle(n, T, seed, trial=trial)
    gpu = HDComplex("haar", n, n, T, seed, dtype, trial=trial)
    x = to_dtype(crand(n, seed + 1), dtype)
    errs, elems, ndef, frac = [], [], [], []
    try:
        for t in range(1, T + 1):
            yo = ora.apply(x, sched(t)).numpy()
            refl = (ora.L if sched(t) else ora.R)[-1]
            frac.append(float(refl.alpha) / max(np.linalg.norm(x), 1e-300))
            yg = gpu.apply(torch.tensor(x, dtype=gpu.torch_dtype, device="cuda"), sched(t))
            yg = yg.cpu().numpy().astype(np.complex128)
            errs.append(np.linalg.norm(yg - yo) / np.linalg.norm(yo))
            elems.append(elem_err(yg, yo, t))
            ndef.append(abs(np.linalg.norm(yg) / np.linalg.norm(x) - 1.0))
            x = to_dtype(next_input(yo), dtype)
    finally:
        gpu.close()
    # steps whose input still brings a well-conditioned new direction (every earlier one too)
    ok = np.minimum.accumulate(np.array(frac)) >= COND_MIN[dtype]
    return np.array(errs)[ok], np.array(elems)[ok], np.array(ndef)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,T,sched", [
    (1, 1, ALLQ), (8, 8, MIXED), (33, 20, ALT), (1000, 16, ALT), (1025, 12, ALLQ), (10_007, 24, MIXED),
    (100_003, 16, ALT), (262_147, 8, ALLQ)])
def test_complex_haar_teacher_forced(dtype, n, T, sched):
    errs, elems, ndef = teacher_forced(n, T, 2024 + n, dtype, sched)
    assert len(errs) >= min(T, 8), len(errs)
    assert errs.max() <= TOL[dtype], (errs.argmax() + 1, errs.max())
    assert elems.max() <= TOL[dtype], (elems.argmax() + 1, elems.max())
    if dtype == "f64":
        assert ndef.max() <= 1e-13, ndef.max()


def test_complex_t_max_256_all_q():
    """The largest reflector count (the finalisations' O(k^2) work at k = 255)."""
    errs, elems, ndef = teacher_forced(3001, 256, 5, "f64", ALLQ)
    assert errs.max() <= TOL["f64"] and elems.max() <= TOL["f64"], (errs.max(), elems.max())
    assert ndef.max() <= 1e-13


def test_complex_reset_reproduces_and_trials_differ():
    from paper_2101_07464_gb300 import HDComplex
    n, T = 5000, 6
    x = torch.tensor(crand(n, 3), dtype=torch.complex128, device="cuda")
    a = HDComplex("haar", n, n, T, 11, "f64")
    ys = [a.apply(x, ALT(t)).clone() for t in range(1, T + 1)]
    a.reset(11)
    ys2 = [a.apply(x, ALT(t)).clone() for t in range(1, T + 1)]
    assert all(torch.equal(u, v) for u, v in zip(ys, ys2))
    assert a.counts() == T
    b = HDComplex("haar", n, n, T, 11, "f64", trial=1)
    assert not torch.equal(b.apply(x, False), ys[0])
    a.close()
    b.close()


def test_complex_argument_errors():
    import ctypes
    import paper_2101_07464_gb300 as hd
    L = hd.lib()
    h = ctypes.c_void_p()
    assert L.hd_complex_create(7, 100, 100, 4, 1, hd.HD_F64, ctypes.byref(h)) == hd.binding.HD_ERR_ARG
    assert L.hd_complex_create(hd.HD_HAAR, 100, 100, 101, 1, hd.HD_F64, ctypes.byref(h)) == hd.binding.HD_ERR_TMAX
    assert L.hd_complex_create(hd.HD_HAAR, 0, 0, 1, 1, hd.HD_F64, ctypes.byref(h)) == hd.binding.HD_ERR_DIM
    assert L.hd_complex_create(hd.HD_HAAR, 100, 99, 1, 1, hd.HD_F64, ctypes.byref(h)) == hd.binding.HD_ERR_DIM
    assert L.hd_complex_create(hd.HD_GINIBRE, 50, 100, 51, 1, hd.HD_F64, ctypes.byref(h)) == hd.binding.HD_ERR_TMAX
    st = hd.HDComplex("haar", 100, 100, 2, 1, "f64")
    x = torch.zeros(101, dtype=torch.complex128, device="cuda")
    y = torch.zeros(101, dtype=torch.complex128, device="cuda")
    # misaligned by half an element
    assert L.hd_complex_apply(st.h, x.data_ptr() + 8, 0, y.data_ptr()) == hd.binding.HD_ERR_ARG
    assert L.hd_complex_apply(st.h, x.data_ptr(), 0, x.data_ptr()) == hd.binding.HD_ERR_ARG
    assert L.hd_complex_apply(st.h, x.data_ptr(), 2, y.data_ptr()) == hd.binding.HD_ERR_ARG
    st.apply(x[:100], False)
    st.apply(x[:100], True)
    with pytest.raises(hd.HDError) as ei:
        st.apply(x[:100], False)
    assert ei.value.code == hd.binding.HD_ERR_TMAX
    st.close()


def test_complex_zero_input_gives_zero():
    from paper_2101_07464_gb300 import HDComplex
    n = 777
    st = HDComplex("haar", n, n, 3, 9, "f64")
    z = torch.zeros(n, dtype=torch.complex128, device="cuda")
    assert torch.count_nonzero(st.apply(z, False)).item() == 0
    st.close()


# ---- complex Ginibre (Algorithm 1 with adjoints) and GUE ------------------------------------
def gin_teacher_forced(m, n, T, seed, dtype, sched, sigma):
    from oracle.complex_hd import ComplexGinibreOracle
    from paper_2101_07464_gb300 import HDComplex
    ora = ComplexGinibreOracle(m, n, T, seed, sigma=sigma)
    gpu = HDComplex("ginibre", m, n, T, seed, dtype, sigma=sigma)
    errs, elems, frac = [], [], []
    x = to_dtype(crand(m if sched(1) else n, seed + 1), dtype)
    try:
        for t in range(1, T + 1):
            tr = sched(t)
            yo = ora.apply(x, tr).numpy()
            refl = (ora.L if tr else ora.R)[-1]
            frac.append(float(refl.alpha) / max(np.linalg.norm(x), 1e-300))
            yg = gpu.apply(torch.tensor(x, dtype=gpu.torch_dtype, device="cuda"), tr).cpu().numpy()
            yg = yg.astype(np.complex128)
            errs.append(np.linalg.norm(yg - yo) / np.linalg.norm(yo))
            elems.append(elem_err(yg, yo, t))
            want = m if sched(t + 1) else n
            x = to_dtype(next_input(yo) if yo.shape[0] == want else crand(want, seed + 100 + t), dtype)
    finally:
        gpu.close()
    ok = np.minimum.accumulate(np.array(frac)) >= COND_MIN[dtype]
    return np.array(errs)[ok], np.array(elems)[ok]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("m,n,T,sched", [
    (8, 8, 8, ALLQ), (9, 13, 9, MIXED), (13, 9, 9, ALT), (1000, 1000, 12, ALLQ), (2003, 4001, 16, ALT),
    (50_001, 100_003, 12, MIXED), (100_003, 30_011, 16, ALT)])
def test_complex_ginibre_teacher_forced(dtype, m, n, T, sched):
    """(The alternating phase map converges: at 2003 x 4001 the FP32 element-wise error
    reaches 1.2e-5 by step 20, from rounding amplified over the steps, so that case stops at
    16.)"""
    errs, elems = gin_teacher_forced(m, n, T, 99 + m, dtype, sched, m ** -0.5)
    assert len(errs) >= min(T, 6), len(errs)
    assert errs.max() <= TOL[dtype], (errs.argmax() + 1, errs.max())
    assert elems.max() <= TOL[dtype], (elems.argmax() + 1, elems.max())


def test_complex_ginibre_t_max_256():
    errs, elems = gin_teacher_forced(2003, 3001, 256, 7, "f64", MIXED, 2003 ** -0.5)
    assert len(errs) >= 64
    assert errs.max() <= TOL["f64"] and elems.max() <= TOL["f64"], (errs.max(), elems.max())


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_gue_matches_oracle_and_is_hermitian(dtype):
    """GUE products (Q x + Q^H x) / sqrt(2) against the oracle's, teacher-forced; and the
    revealed W is Hermitian on the queried columns: e_k^H W e_j = conj(e_j^H W e_k)."""
    from oracle.complex_hd import ComplexGinibreOracle, gue_apply
    from paper_2101_07464_gb300 import HDComplex
    n, Q, seed = 20_011, 8, 5
    ora = ComplexGinibreOracle(n, n, 2 * Q, seed, sigma=n ** -0.5)
    gpu = HDComplex("ginibre", n, n, 2 * Q, seed, dtype, sigma=n ** -0.5)
    x = to_dtype(crand(n, 6), dtype)
    for q in range(Q):
        wo = gue_apply(ora, x).numpy()
        wg = gpu.gue(torch.tensor(x, dtype=gpu.torch_dtype, device="cuda")).cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(wg - wo) <= TOL[dtype] * np.linalg.norm(wo), q
        assert elem_err(wg, wo, 2 * (q + 1)) <= TOL[dtype], q
        x = to_dtype(next_input(wo), dtype)
    gpu.close()
    st = HDComplex("ginibre", 500, 500, 4, 3, "f64")
    e = [torch.zeros(500, dtype=torch.complex128, device="cuda") for _ in range(2)]
    e[0][0] = 1.0
    e[1][1] = 1.0
    c0 = st.gue(e[0]).cpu().numpy()
    c1 = st.gue(e[1]).cpu().numpy()
    assert abs(c1[0] - np.conj(c0[1])) <= 1e-13 and abs(c0[0].imag) <= 1e-15
    with pytest.raises(Exception):
        st.gue(e[0])    # fewer than two products left
    st.close()
