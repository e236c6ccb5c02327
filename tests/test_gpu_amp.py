"""hd_run with HD_DYN_AMP on batched Gin states: every trial's AMP trajectory (product 1 =
Q beta, then Q^T z / Q x alternating, soft threshold a ||z|| / sqrt(m), Onsager term) equals
the oracle's AMP on that trial's own Householder Dice oracle (free-running).

* FP64: final x per trial to 1e-9 relative (threshold decisions are identical unless a
  component lands within rounding of the threshold).
* FP32: final MSE per trial to 1e-3 relative.
* Per-trial entry scales sigma_i = 1/sqrt(m_i) (hd_set_trial_sigmas), uneven sizes, one
  CUDA graph; graph and stream replays give identical results.
"""
import numpy as np
import pytest

import synth
from oracle.dynamics import amp as oracle_amp
from oracle.hd import GinibreOracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_gpu(ns, ms, T, seed, dtype, graph, base_trial=0, reps=1):
    import paper_2101_07464_gb300 as hd
    tdt = torch.float64 if dtype == "f64" else torch.float32
    b = hd.HDBatch("ginibre", ms, ns, T, seed, dtype, trial=base_trial)
    b.set_trial_sigmas([m ** -0.5 for m in ms])
    beta = np.concatenate([synth.bernoulli_gauss(n, seed, trial=i) for i, n in enumerate(ns)])
    w = np.concatenate([synth.noise(m, seed, trial=i) for i, m in enumerate(ms)])
    bt = torch.tensor(beta, dtype=tdt, device="cuda")
    wt = torch.tensor(w, dtype=tdt, device="cuda")
    out = torch.empty(int(b.off_n[-1]), dtype=tdt, device="cuda")
    flags = [t % 2 == 0 for t in range(1, T + 1)]
    spec = hd.make_run_spec(flags, "amp", 1.1, use_graph=graph, aux=wt)
    outs = []
    for _ in range(reps):
        hd.hd_run(b.h, spec, bt, out)
        torch.cuda.synchronize()
        outs.append(out.double().cpu().numpy().copy())
    off = b.off_n.copy()
    b.close()
    return outs, off, beta


def run_oracle(n, m, T, seed, trial):
    st = GinibreOracle(m, n, T, seed, trial=trial, sigma=m ** -0.5)
    beta = synth.bernoulli_gauss(n, seed, trial=trial)
    w = synth.noise(m, seed, trial=trial)
    xs, _ = oracle_amp(st, beta, w, T)
    return xs[-1], beta


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_amp_matches_oracle(dtype):
    ns = [1200, 5003, 30_011, 2047]
    ms = [n // 2 for n in ns]
    T, seed = 30, 21
    outs, off, beta = run_gpu(ns, ms, T, seed, dtype, graph=True, reps=2)
    np.testing.assert_array_equal(outs[0], outs[1])   # graph replay is deterministic
    for i, (n, m) in enumerate(zip(ns, ms)):
        xo, bo = run_oracle(n, m, T, seed, i)
        xg = outs[0][off[i]:off[i + 1]]
        if dtype == "f64":
            assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo), i
        else:
            mse_g = np.mean((xg - bo) ** 2)
            mse_o = np.mean((xo - bo) ** 2)
            assert abs(mse_g - mse_o) <= 1e-3 * mse_o, (i, mse_g, mse_o)


def test_amp_graph_and_stream_agree_and_errors():
    import paper_2101_07464_gb300 as hd
    ns = [3001, 4000]
    ms = [1500, 2000]
    a, _, _ = run_gpu(ns, ms, 12, 5, "f32", graph=False)
    b, _, _ = run_gpu(ns, ms, 12, 5, "f32", graph=True)
    np.testing.assert_array_equal(a[0], b[0])
    st = hd.HDBatch("ginibre", ms, ns, 4, 1, "f32")
    x = torch.zeros(sum(ns), dtype=torch.float32, device="cuda")
    w = torch.zeros(sum(ms), dtype=torch.float32, device="cuda")
    with pytest.raises(hd.HDError) as ei:   # AMP needs Q, Q^T, Q, ...
        hd.hd_run(st.h, hd.make_run_spec([True, False], "amp", 1.1, aux=w), x, x)
    assert ei.value.code == 1
    with pytest.raises(hd.HDError) as ei:   # and the noise vector
        hd.hd_run(st.h, hd.make_run_spec([False, True], "amp", 1.1), x, x)
    assert ei.value.code == 1
    st.close()
