"""Batched states: `count` independent trials advanced by one launch per sweep.

* Every trial of a batch matches its own oracle (trial word = base + i), teacher-forced, to the
  single-trial tolerances, with uneven dimensions (one CTA .. many CTAs, T = n, ragged tails)
  and rectangular Ginibre trials of both shapes.
* A batch of one is the single-trial state, bit for bit.
* hd_run on a batch equals hd_apply on the same batch driven step by step, bit for bit.
"""
import numpy as np
import pytest

import synth
from gpu_util import TOL
from oracle.hd import make_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALT = lambda t: t % 2 == 0
MIXED = lambda t: t in (2, 3, 7, 8, 9)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batched_teacher_forced(ens, ms, ns, T, seed, dtype, sched, base_trial=5):
    from paper_2101_07464_gb300 import HDBatch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    count = len(ns)
    sig = [1.0 if ens == "haar" else 0.7] * count
    b = HDBatch(ens, ms, ns, T, seed, dtype, sigma=sig[0], trial=base_trial)
    ora = [make_oracle(ens, ms[i], ns[i], T, seed, trial=base_trial + i, sigma=sig[i])
           for i in range(count)]
    xs = [synth.x1(ms[i] if sched(1) else ns[i], seed, trial=i) for i in range(count)]
    errs = np.zeros((count, T))
    try:
        for t in range(1, T + 1):
            tr = sched(t)
            xs = [np.asarray(x, dtype=np.float64) for x in xs]
            if dtype == "f32":
                xs = [x.astype(np.float32).astype(np.float64) for x in xs]
            y = b.apply(torch.tensor(np.concatenate(xs), dtype=tdt, device="cuda"), tr)
            y = y.double().cpu().numpy()
            off = b.off_n if tr else b.off_m
            nxt = []
            for i in range(count):
                yo = ora[i].apply(xs[i], tr).numpy()
                yg = y[off[i]:off[i + 1]]
                den = np.linalg.norm(yo)
                errs[i, t - 1] = np.linalg.norm(yg - yo) / den if den > 0 else np.linalg.norm(yg)
                want = ms[i] if sched(t + 1) else ns[i]
                nxt.append(np.tanh(yo) if yo.shape[0] == want else synth.x1(want, seed, trial=100 * t + i))
            xs = nxt
    finally:
        b.close()
    return errs


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("ns,sched", [
    ([1000, 5003, 17, 100_003, 12, 40_000], ALT),
    ([262_147, 33, 8191], MIXED)])
def test_batched_haar_per_trial(dtype, ns, sched):
    errs = _batched_teacher_forced("haar", ns, ns, 12, 321, dtype, sched)
    assert errs.max() <= TOL[dtype], errs


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_ginibre_per_trial(dtype):
    ms = [13, 2003, 50_001, 10]
    ns = [11, 4001, 30_011, 10]
    errs = _batched_teacher_forced("ginibre", ms, ns, 10, 654, dtype, ALT)
    assert errs.max() <= TOL[dtype], errs


@pytest.mark.parametrize("ens", ["haar", "ginibre"])
def test_batch_of_one_is_single_state(ens):
    from paper_2101_07464_gb300 import HD, HDBatch
    m, n, T = 3001, 5003, 8
    if ens == "haar":
        m = n
    st = HD(ens, m, n, T, 17, "f64", sigma=0.3, trial=4)
    b = HDBatch(ens, [m], [n], T, 17, "f64", sigma=0.3, trial=4)
    x = torch.tensor(synth.x1(n, 2), dtype=torch.float64, device="cuda")
    for t in range(1, T + 1):
        tr = ALT(t)
        ya, yb = st.apply(x, tr), b.apply(x, tr)
        assert torch.equal(ya, yb), t
        want = m if ALT(t + 1) else n
        x = torch.tanh(ya) if ya.numel() == want else torch.tensor(synth.x1(want, t), dtype=torch.float64, device="cuda")
    st.close()
    b.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("graph", [False, True])
def test_batched_run_matches_apply(dtype, graph):
    import paper_2101_07464_gb300 as hd
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ns = [10_007, 31, 65_536, 4099]
    T, a = 14, 0.5
    flags = [ALT(t) for t in range(1, T + 1)]
    x1 = torch.tensor(np.concatenate([synth.x1(n, 8, trial=i) for i, n in enumerate(ns)]),
                      dtype=tdt, device="cuda")
    b = hd.HDBatch("haar", ns, ns, T, 8, dtype, trial=2)
    hd.hd_set_engine(b.h, no_fuse=True)   # bit-exact comparison: the unfused path
    x, xp = x1.clone(), torch.zeros_like(x1)
    for t in range(T):
        y = b.apply(x, flags[t])
        x, xp = torch.sign(y) + a * xp, x
    b.reset(8)
    out = torch.empty_like(x1)
    spec = hd.make_run_spec(flags, "sign_mem", a, use_graph=graph)
    for rep in range(2):
        hd.hd_run(b.h, spec, x1, out)
        torch.cuda.synchronize()
        assert torch.equal(out, x), (out - x).abs().max().item()
    b.close()


def test_batched_argument_checks():
    import paper_2101_07464_gb300 as hd
    with pytest.raises(hd.HDError) as ei:
        hd.HDBatch("haar", [10, 20], [10, 21], 4, 1, "f64")   # Haar needs m == n
    assert ei.value.code in (1, 2)
    with pytest.raises(ValueError):
        hd.HDBatch("ginibre", [10, 20], [10], 4, 1, "f64")
    b = hd.HDBatch("ginibre", [10, 20], [30, 40], 4, 1, "f64")
    assert list(b.off_n) == [0, 30, 70] and list(b.off_m) == [0, 10, 30]
    tr = hd.make_run_spec([False, False], "tanh")   # Q then Q: packed 30 != 70 per trial
    with pytest.raises(hd.HDError) as ei:
        hd.hd_run(b.h, tr, torch.zeros(70, dtype=torch.float64, device="cuda"),
                  torch.zeros(70, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 2
    nt = hd.make_run_spec([False], "norm_tanh")   # one norm per trial is not offered for batches
    with pytest.raises(hd.HDError) as ei:
        hd.hd_run(b.h, nt, torch.zeros(70, dtype=torch.float64, device="cuda"),
                  torch.zeros(70, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 1
    b.close()


def test_batched_fused_run_matches_apply():
    """Fused alternating trajectory on a batch (FP64, sign dynamics): per trial equal to the
    step-by-step products up to the dots' summation order.  Every trial has n >= 333: with
    n <= 257 this schedule revisits sign vectors exactly (x_t falls in the span the earlier
    reflectors fix, alpha_t = 0 in exact arithmetic, reading A15), and the reflector built from
    that rounding-level remainder differs between any two summation orders."""
    import paper_2101_07464_gb300 as hd
    ns = [10_007, 333, 65_536, 4099]
    T, a = 14, 0.5
    flags = [ALT(t) for t in range(1, T + 1)]
    x1 = torch.tensor(np.concatenate([synth.x1(n, 9, trial=i) for i, n in enumerate(ns)]),
                      dtype=torch.float64, device="cuda")
    b = hd.HDBatch("haar", ns, ns, T, 9, "f64", trial=3)
    x, xp = x1.clone(), torch.zeros_like(x1)
    for t in range(T):
        y = b.apply(x, flags[t])
        x, xp = torch.sign(y) + a * xp, x
    b.reset(9)
    out = torch.empty_like(x1)
    hd.hd_run(b.h, hd.make_run_spec(flags, "sign_mem", a, use_graph=True), x1, out)
    torch.cuda.synchronize()
    off = b.off_n
    for i in range(len(ns)):
        xo, xr = out[off[i]:off[i + 1]].double(), x[off[i]:off[i + 1]].double()
        assert (xo - xr).norm().item() <= 1e-12 * xr.norm().item(), i
    b.close()


def test_batched_fused_ginibre_run_matches_apply():
    """Fused alternating trajectory on a batch of rectangular Ginibre trials (FP64, tanh):
    per trial equal to the step-by-step products up to the dots' summation order."""
    import paper_2101_07464_gb300 as hd
    ms = [3001, 40, 20_000]
    ns = [5003, 64, 12_011]
    T = 12
    flags = [ALT(t) for t in range(1, T + 1)]
    x1 = torch.tensor(np.concatenate([synth.x1(n, 4, trial=i) for i, n in enumerate(ns)]),
                      dtype=torch.float64, device="cuda")
    b = hd.HDBatch("ginibre", ms, ns, T, 4, "f64", trial=1)
    b.set_trial_sigmas([m ** -0.5 for m in ms])
    x = x1.clone()
    for t in range(T):
        x = torch.tanh(b.apply(x, flags[t]))
    b.reset(4)
    out = torch.empty(int(b.off_m[-1]) if not flags[-1] else int(b.off_n[-1]), dtype=torch.float64, device="cuda")
    hd.hd_run(b.h, hd.make_run_spec(flags, "tanh", 0.0, use_graph=True), x1, out)
    torch.cuda.synchronize()
    off = b.off_n if flags[-1] else b.off_m
    for i in range(len(ns)):
        xo, xr = out[off[i]:off[i + 1]], x[off[i]:off[i + 1]]
        assert (xo - xr).norm().item() <= 1e-12 * xr.norm().item(), i
    b.close()
