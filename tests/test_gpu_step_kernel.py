"""The step kernel: a fused step of hd_run (update sweep, then the output sweep with f_t and
the next step's dots) as one cooperative launch over all trials of a batch.

* Switched on (hd_set_engine), it is the path hd_run takes: the profile shows T - 1
  step-kernel launches and no separate update or output sweep except in the last step.
* It computes what the two-launch path computes (same sweeps, same per-CTA arithmetic; the
  output sweep may take another stage count, which only reorders FP64 column sums): whole
  trajectories agree to 1e-13 (FP64) and 1e-6 (FP32) relative, per trial.
* Batches with more CTAs in their maps than the GPU holds at once (hundreds of small uneven
  trials, Haar and rectangular Ginibre, and batched AMP): every CTA of the launch walks
  several virtual CTAs, finalises several trials, and waits on several trials' flags.  Per
  trial the result equals the two-launch path, and for a few trials the oracle's trajectory.
* The oracle parity of the benchmarked trajectory (element-wise, teacher-forced, n = 10^6)
  runs through this kernel in test_gpu_trajectory_parity.py.
"""
import numpy as np
import pytest

import synth
from gpu_util import oracle_trajectory
from oracle.dynamics import f_sign_mem, f_tanh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALT = lambda t: t % 2 == 0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(st, flags, dyn, a, x1, out_len, step_kernel, aux=None, profile=False):
    import paper_2101_07464_gb300 as hd
    hd.hd_set_engine(st.h, step_kernel=step_kernel)
    st.reset(st.seed)
    if profile:
        hd.hd_profile_enable(st.h, True)
        hd.hd_profile_read(st.h, clear=True)
    out = torch.empty(out_len, dtype=st.torch_dtype, device="cuda")
    spec = hd.make_run_spec(flags, dyn, a, use_graph=True, aux=aux)
    for _ in range(2):   # capture, then a replay of the captured graph
        hd.hd_run(st.h, spec, x1, out)
    torch.cuda.synchronize()
    hd.hd_sync(st.h)
    prof = None
    if profile:
        prof = hd.hd_profile_read(st.h, clear=True)
        hd.hd_profile_enable(st.h, False)
    return out.double().cpu().numpy(), prof


def _per_trial_close(a, b, off, tol):
    for i in range(len(off) - 1):
        lo, hi = int(off[i]), int(off[i + 1])
        den = np.linalg.norm(b[lo:hi])
        err = np.linalg.norm(a[lo:hi] - b[lo:hi]) / (den if den > 0 else 1.0)
        assert err <= tol, (i, err)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_step_kernel_matches_two_launches(dtype):
    import paper_2101_07464_gb300 as hd
    n, T, seed = 200_003, 20, 5
    st = hd.HD("haar", n, n, T, seed, dtype)
    x1 = torch.tensor(synth.x1(n, seed), dtype=st.torch_dtype, device="cuda")
    flags = [ALT(t) for t in range(1, T + 1)]
    one, prof = _run(st, flags, "sign_mem", 0.5, x1, n, True, profile=True)
    # the events of the last run (a graph replay re-records the captured events): T - 1 fused
    # steps in the step kernel, the last step as an update and an output sweep
    assert prof["step"][1] == T - 1, prof
    assert prof["update"][1] == 1 and prof["output"][1] == 1, prof
    two, prof2 = _run(st, flags, "sign_mem", 0.5, x1, n, False, profile=True)
    assert prof2["step"][1] == 0 and prof2["update"][1] == T, prof2
    st.close()
    _per_trial_close(one, two, [0, n], 1e-13 if dtype == "f64" else 1e-6)


def test_step_kernel_many_virtual_ctas_haar():
    """700 uneven small Haar trials (333 .. 3000 rows: one CTA each in the built-in split, far
    more CTAs than one wave holds), FP64, sign with memory.  (Below about 333 rows this
    schedule revisits sign vectors exactly, alpha_t = 0, and the trajectory is set by rounding:
    reading A15.)"""
    import paper_2101_07464_gb300 as hd
    rng = np.random.default_rng(11)
    ns = [int(v) for v in rng.integers(333, 3001, size=700)]
    T, seed, a, base = 12, 17, 0.5, 3
    st = hd.HDBatch("haar", ns, ns, T, seed, "f64", trial=base)
    x1h = [synth.x1(n, seed, trial=i) for i, n in enumerate(ns)]
    x1 = torch.tensor(np.concatenate(x1h), dtype=torch.float64, device="cuda")
    flags = [ALT(t) for t in range(1, T + 1)]
    L = int(st.off_n[-1])
    one, prof = _run(st, flags, "sign_mem", a, x1, L, True, profile=True)
    assert prof["step"][1] == T - 1, prof
    two, _ = _run(st, flags, "sign_mem", a, x1, L, False)
    off = st.off_n
    st.close()
    _per_trial_close(one, two, off, 1e-13)
    for i in (0, 350, 699):   # the oracle's own trajectories, free-running
        xs, ys, fs = oracle_trajectory("haar", ns[i], ns[i], T, seed, ALT, f_sign_mem, x1h[i], trial=base + i)
        lo, hi = int(off[i]), int(off[i + 1])
        err = np.linalg.norm(one[lo:hi] - fs[-1]) / np.linalg.norm(fs[-1])
        assert err <= 1e-12, (i, err)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_step_kernel_many_virtual_ctas_ginibre(dtype):
    """500 uneven rectangular Ginibre trials (m < n and m > n), alternating tanh."""
    import paper_2101_07464_gb300 as hd
    rng = np.random.default_rng(12)
    ns = [int(v) for v in rng.integers(64, 4000, size=500)]
    ms = [int(v) for v in rng.integers(64, 4000, size=500)]
    T, seed, base = 10, 23, 1
    st = hd.HDBatch("ginibre", ms, ns, T, seed, dtype, trial=base)
    st.set_trial_sigmas([m ** -0.5 for m in ms])
    x1h = [synth.x1(n, seed, trial=i) for i, n in enumerate(ns)]
    x1 = torch.tensor(np.concatenate(x1h), dtype=st.torch_dtype, device="cuda")
    flags = [ALT(t) for t in range(1, T + 1)]
    L = int(st.off_m[-1]) if not flags[-1] else int(st.off_n[-1])
    one, prof = _run(st, flags, "tanh", 0.0, x1, L, True, profile=True)
    assert prof["step"][1] == T - 1, prof
    two, _ = _run(st, flags, "tanh", 0.0, x1, L, False)
    off = st.off_n if flags[-1] else st.off_m
    st.close()
    _per_trial_close(one, two, off, 1e-13 if dtype == "f64" else 1e-6)
    if dtype == "f64":
        for i in (0, 499):
            xs, ys, fs = oracle_trajectory("ginibre", ms[i], ns[i], T, seed, ALT, f_tanh, x1h[i],
                                           sigma=ms[i] ** -0.5, trial=base + i)
            lo, hi = int(off[i]), int(off[i + 1])
            err = np.linalg.norm(one[lo:hi] - fs[-1]) / np.linalg.norm(fs[-1])
            assert err <= 1e-12, (i, err)


def test_step_kernel_batched_amp_many_trials():
    """Batched AMP over 600 uneven trials of Gin(n/2, n): the fused AMP sweep inside the step
    kernel, with its per-trial norms and counts, equals the two-launch path per trial."""
    import paper_2101_07464_gb300 as hd
    rng = np.random.default_rng(13)
    ns = [int(v) for v in rng.integers(200, 6000, size=600)]
    ms = [n // 2 for n in ns]
    T, seed = 16, 29
    st = hd.HDBatch("ginibre", ms, ns, T, seed, "f32")
    st.set_trial_sigmas([m ** -0.5 for m in ms])
    beta = torch.tensor(np.concatenate([synth.bernoulli_gauss(n, seed, trial=i) for i, n in enumerate(ns)]),
                        dtype=torch.float32, device="cuda")
    w = torch.tensor(np.concatenate([synth.noise(m, seed, trial=i) for i, m in enumerate(ms)]),
                     dtype=torch.float32, device="cuda")
    flags = [ALT(t) for t in range(1, T + 1)]
    L = int(st.off_n[-1]) if flags[-1] else int(st.off_m[-1])
    one, prof = _run(st, flags, "amp", 1.1, beta, L, True, aux=w, profile=True)
    assert prof["step"][1] == T - 1, prof
    two, _ = _run(st, flags, "amp", 1.1, beta, L, False, aux=w)
    off = st.off_n if flags[-1] else st.off_m
    st.close()
    _per_trial_close(one, two, off, 1e-5)
