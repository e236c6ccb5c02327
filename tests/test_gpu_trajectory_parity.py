"""Oracle parity of the trajectory path that bench.py times (hd_run, one CUDA graph, launch
shapes from hd_autotune), element by element and step by step.

For Q / Q^T alternating schedules with an elementwise f_t, hd_run folds f_t and the next
step's dot sweep into each output sweep and never stores y_t.  The run spec's records expose
it: y_record receives every y_t from inside the fused sweep, x_record the library's own f_t
result, and x_given feeds the oracle's x_{t+1} back as the next product's input (teacher
forcing, the per-step protocol of reading A13: both sides apply M_t to the same x_t).

* Haar(n), n = 10^6, T = 100, x_{t+1} = sign(y_t) + 0.5 x_{t-1} (the benchmarked workload),
  FP64 and FP32: per step the norm error ||y_gpu - y_ora|| / ||y_ora|| <= tol and the
  element-wise error <= tol, tol = 1e-12 (FP64) / 1e-5 (FP32).  Element-wise means
  |y_gpu,i - y_ora,i| relative to max_j |y_ora,j|, except on the t pivot rows fixed by the
  reflectors so far, which are relative to ||y_ora|| (gpu_util.elem_err: the oracle's own
  rounding there scales with the vector norm).  About 103 sub-tiles of 32 rows per CTA; both
  stacks reach k = 99 columns.  The schedule is well conditioned at this n: the oracle moved
  by one rounding of x_1 stays at the rounding level through T = 100 (its outputs then
  differ by at most 2e-14 relative at n = 10^5), so any two correct implementations agree to
  these tolerances.
* The library's own f_t results agree with f of the oracle's y_t; a sign decision whose
  argument lies within the tolerance of zero may go either way.
* FP64 free-running (no teacher): the whole trajectory follows the oracle's to 1e-12.
* Ginibre, rectangular, alternating tanh (the fused Ginibre output sweep).
* Batched AMP, the fused AMP sweep: products and updates (soft threshold, Onsager term, the
  per-trial norms and counts) against the oracle's AMP, teacher-forced, element by element.
"""
import numpy as np
import pytest

import synth
from gpu_util import TOL, elem_err, f32_cast, oracle_trajectory
from oracle.dynamics import amp_trace, f_sign_mem, f_tanh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALT = lambda t: t % 2 == 0   # Q at odd t, Q^T at even t


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rows(vs, L, tdt):
    out = torch.zeros((len(vs), L), dtype=tdt, device="cuda")
    for i, v in enumerate(vs):
        out[i, :v.shape[0]] = torch.tensor(v, dtype=tdt)
    return out


def run_recorded(st, flags, dyn, a, x1, L, given=None, autotune=False, graph=True, aux=None):
    """hd_run with y_record / x_record (and x_given when given); returns both records (host)."""
    import paper_2101_07464_gb300 as hd
    T = len(flags)
    tdt = st.torch_dtype
    yrec = torch.zeros((T, L), dtype=tdt, device="cuda")
    xrec = torch.zeros((T, L), dtype=tdt, device="cuda")
    out = torch.empty(L, dtype=tdt, device="cuda")
    if autotune:
        st.autotune(flags, dyn, x1, a=a, reps=1, aux=aux)
    spec = hd.make_run_spec(flags, dyn, a, use_graph=graph, aux=aux, y_record=yrec, x_record=xrec,
                            x_given=given)
    for _ in range(2 if graph else 1):   # capture, then a replay of the captured graph
        hd.hd_run(st.h, spec, x1, out)
    torch.cuda.synchronize()
    hd.hd_sync(st.h)   # raises on a device-side error
    return yrec.double().cpu().numpy(), xrec.double().cpu().numpy()


N_HEAD, T_HEAD, SEED_HEAD = 1_000_000, 100, 12


@pytest.fixture(scope="module")
def headline_oracle():
    """The oracle's sign-with-memory trajectories: FP64 inputs, and inputs rounded to FP32."""
    x1 = synth.x1(N_HEAD, SEED_HEAD)
    return {"f64": oracle_trajectory("haar", N_HEAD, N_HEAD, T_HEAD, SEED_HEAD, ALT, f_sign_mem, x1),
            "f32": oracle_trajectory("haar", N_HEAD, N_HEAD, T_HEAD, SEED_HEAD, ALT, f_sign_mem, x1,
                                     cast=f32_cast)}


def check_sign_records(xs, ys, fs, yrec, xrec, tol):
    """Per step t: y_t element-wise and in norm; f's result sign(y_t) + 0.5 x_{t-1}
    element-wise, except where y_t's entry is within the tolerance of zero: there the sign
    may go either way, so the entry must be 0.5 x_{t-1} plus -1, 0 or 1."""
    for i in range(len(ys)):
        y = ys[i]
        e = elem_err(yrec[i], y, i + 1)
        en = np.linalg.norm(yrec[i] - y) / np.linalg.norm(y)
        assert e <= tol and en <= tol, (i + 1, e, en)
        amb = np.abs(y) <= tol * np.abs(y).max()
        amb[:i + 1] |= np.abs(y[:i + 1]) <= tol * np.linalg.norm(y)
        d = np.abs(xrec[i] - fs[i])
        d[amb] = 0.0
        d[:i + 1] *= np.abs(fs[i]).max() / np.linalg.norm(fs[i])
        ex = d.max() / np.abs(fs[i]).max()
        assert ex <= tol, (i + 1, ex)
        if amb.any():
            xprev = xs[i - 1][amb] if i >= 1 else 0.0
            jump = xrec[i][amb] - 0.5 * xprev
            assert np.all(np.min(np.abs(jump[:, None] - np.array([-1.0, 0.0, 1.0])[None, :]), axis=1) <= 1e-6)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_headline_fused_trajectory_teacher_forced(headline_oracle, dtype):
    import paper_2101_07464_gb300 as hd
    xs, ys, fs = headline_oracle[dtype]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    flags = [ALT(t) for t in range(1, T_HEAD + 1)]
    st = hd.HD("haar", N_HEAD, N_HEAD, T_HEAD, SEED_HEAD, dtype)
    x1 = torch.tensor(xs[0], dtype=tdt, device="cuda")
    given = _rows(xs[1:] + [xs[-1]], N_HEAD, tdt)   # row t-1 = x_{t+1}; row T-1 is not read
    yrec, xrec = run_recorded(st, flags, "sign_mem", 0.5, x1, N_HEAD, given=given, autotune=True)
    st.close()
    check_sign_records(xs, ys, fs, yrec, xrec, TOL[dtype])


def test_headline_fused_trajectory_free_running_f64(headline_oracle):
    """No teacher: the GPU applies its own f_t; FP64 sign decisions far from zero agree, so
    the whole trajectory stays on the oracle's to 1e-12."""
    import paper_2101_07464_gb300 as hd
    xs, ys, fs = headline_oracle["f64"]
    flags = [ALT(t) for t in range(1, T_HEAD + 1)]
    st = hd.HD("haar", N_HEAD, N_HEAD, T_HEAD, SEED_HEAD, "f64")
    x1 = torch.tensor(xs[0], dtype=torch.float64, device="cuda")
    yrec, xrec = run_recorded(st, flags, "sign_mem", 0.5, x1, N_HEAD)
    st.close()
    for t in range(T_HEAD):
        assert elem_err(yrec[t], ys[t], t + 1) <= 1e-12, (t + 1, elem_err(yrec[t], ys[t], t + 1))
        assert elem_err(xrec[t], fs[t], t + 1) <= 1e-12, (t + 1, elem_err(xrec[t], fs[t], t + 1))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fused_ginibre_rectangular_teacher_forced(dtype):
    import paper_2101_07464_gb300 as hd
    m, n, T, seed = 131_101, 262_147, 64, 5
    sigma = m ** -0.5
    tdt = torch.float64 if dtype == "f64" else torch.float32
    cast = f32_cast if dtype == "f32" else None
    xs, ys, fs = oracle_trajectory("ginibre", m, n, T, seed, ALT, f_tanh, synth.x1(n, seed), sigma=sigma,
                                   cast=cast)
    L = max(m, n)
    flags = [ALT(t) for t in range(1, T + 1)]
    st = hd.HD("ginibre", m, n, T, seed, dtype, sigma=sigma)
    given = _rows(xs[1:] + [xs[-1]], L, tdt)
    yrec, xrec = run_recorded(st, flags, "tanh", 0.0, torch.tensor(xs[0], dtype=tdt, device="cuda"), L,
                              given=given)
    st.close()
    tol = TOL[dtype]
    for t in range(T):
        d = ys[t].shape[0]
        assert elem_err(yrec[t, :d], ys[t], t + 1) <= tol, (t + 1, elem_err(yrec[t, :d], ys[t], t + 1))
        assert elem_err(xrec[t, :d], fs[t], t + 1) <= tol, (t + 1, elem_err(xrec[t, :d], fs[t], t + 1))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_amp_teacher_forced_elementwise(dtype):
    """Every trial's products y_t and AMP updates (z^0, x^1, z^1, ...) computed by the fused
    AMP sweep from the oracle's previous AMP vectors, against the oracle's, per trial and
    per step, element by element."""
    import paper_2101_07464_gb300 as hd
    ns = [1200, 5003, 30_011, 100_000, 2047]
    ms = [n // 2 for n in ns]
    T, seed = 30, 21
    tdt = torch.float64 if dtype == "f64" else torch.float32
    cast = f32_cast if dtype == "f32" else None
    from oracle.hd import GinibreOracle
    traces = []
    for i, (n, m) in enumerate(zip(ns, ms)):
        ora = GinibreOracle(m, n, T, seed, trial=i, sigma=m ** -0.5)
        beta = synth.bernoulli_gauss(n, seed, trial=i)
        w = synth.noise(m, seed, trial=i)
        if cast is not None:
            beta, w = cast(beta), cast(w)
        traces.append((beta, w, amp_trace(ora, beta, w, T, cast=cast)))
    b = hd.HDBatch("ginibre", ms, ns, T, seed, dtype)
    b.set_trial_sigmas([m ** -0.5 for m in ms])
    off_n, off_m = b.off_n, b.off_m
    L = int(max(off_n[-1], off_m[-1]))
    beta = torch.tensor(np.concatenate([tr[0] for tr in traces]), dtype=tdt, device="cuda")
    wv = torch.tensor(np.concatenate([tr[1] for tr in traces]), dtype=tdt, device="cuda")
    given = torch.zeros((T, L), dtype=tdt, device="cuda")
    for t in range(1, T):   # the vector product t+1 consumes: z^k after a Q step, x^k after Q^T
        off = off_n if t % 2 == 0 else off_m
        row = np.concatenate([tr[2]["used"][t - 1] for tr in traces])
        assert row.shape[0] == off[-1]
        given[t - 1, :row.shape[0]] = torch.tensor(row, dtype=tdt)
    flags = [ALT(t) for t in range(1, T + 1)]
    yrec, xrec = run_recorded(b, flags, "amp", 1.1, beta, L, given=given, aux=wv)
    b.close()
    tol = TOL[dtype]
    for t in range(1, T + 1):
        out_off = off_n if t % 2 == 0 else off_m
        for i, tr in enumerate(traces):
            lo, hi = int(out_off[i]), int(out_off[i + 1])
            y_o = tr[2]["products"][t - 1]
            v_o = tr[2]["updates"][t - 1]
            assert elem_err(yrec[t - 1, lo:hi], y_o, t) <= tol, (t, i, elem_err(yrec[t - 1, lo:hi], y_o, t))
            assert elem_err(xrec[t - 1, lo:hi], v_o, t) <= tol, (t, i, elem_err(xrec[t - 1, lo:hi], v_o, t))


def test_record_argument_checks():
    import paper_2101_07464_gb300 as hd
    n, T = 1000, 4
    st = hd.HD("haar", n, n, T, 1, "f64")
    short = torch.zeros((T, n - 1), dtype=torch.float64, device="cuda")
    spec = hd.make_run_spec([ALT(t) for t in range(1, T + 1)], "tanh", y_record=short)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(hd.HDError) as ei:   # rows shorter than the vectors
        hd.hd_run(st.h, spec, x, x.clone())
    assert ei.value.code == hd.binding.HD_ERR_ARG
    st.close()
