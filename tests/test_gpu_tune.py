"""Launch-shape tuning (hd_autotune, hd_set_tuning, hd_get_tuning, hd_get_map_options).

* Every forced (warps per CTA, stages per warp) shape gives the oracle's products (teacher
  forced, FP64 1e-12, FP32 1e-5), on the step-by-step path (dot, update and output sweeps) and
  on the fused trajectory path (update and fused output sweeps).
* Every candidate CTA split gives the oracle's products (single trial) and the built-in
  split's products to rounding (batch of unequal trials).
* hd_autotune leaves the state reset, writes valid words, changes results only by rounding,
  and its choice is taken over by a new state of the same shape; hd_set_tuning rejects bad
  words and [] restores the built-in rules.
"""
import numpy as np
import pytest

import synth
from gpu_util import TOL, teacher_forced

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS, BUCKETS = 6, 11
ALT = lambda t: t % 2 == 0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def forcing(W, nb, opt=0):
    return [1, opt] + [W, nb] * (KINDS * BUCKETS)


SHAPES = [(1, 1), (1, 8), (2, 4), (4, 2), (4, 8), (8, 8)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("W,nb", SHAPES)
@pytest.mark.parametrize("ens,m,n", [("haar", 20_011, 20_011), ("ginibre", 9001, 15_013)])
def test_forced_shape_teacher_forced(dtype, W, nb, ens, m, n):
    sigma = 1.0 if ens == "haar" else m ** -0.5
    errs = teacher_forced(ens, m, n, 12, seed=31 + W * 10 + nb, dtype=dtype, schedule=ALT,
                          sigma=sigma, setup=lambda g: g.set_tuning(forcing(W, nb)))
    assert errs.max() <= TOL[dtype], errs


def _manual_tanh(ens, m, n, T, seed, dtype, sigma):
    from paper_2101_07464_gb300 import HD
    tdt = torch.float64 if dtype == "f64" else torch.float32
    st = HD(ens, m, n, T, seed, dtype, sigma=sigma)
    x = torch.tensor(synth.x1(n, seed), dtype=tdt, device="cuda")
    for t in range(1, T + 1):
        x = torch.tanh(st.apply(x, ALT(t)))
    st.close()
    return x


@pytest.mark.parametrize("W,nb", [(1, 2), (2, 8), (4, 1), (8, 4)])
@pytest.mark.parametrize("ens,m,n,dtype", [("haar", 30_011, 30_011, "f64"),
                                           ("ginibre", 12_007, 20_011, "f32")])
def test_forced_shape_fused_run(W, nb, ens, m, n, dtype):
    import paper_2101_07464_gb300 as hd
    T = 14
    sigma = 1.0 if ens == "haar" else m ** -0.5
    ref = _manual_tanh(ens, m, n, T, 3, dtype, sigma)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    st = hd.HD(ens, m, n, T, 3, dtype, sigma=sigma)
    st.set_tuning(forcing(W, nb))
    spec = hd.make_run_spec([ALT(t) for t in range(1, T + 1)], "tanh", use_graph=True)
    x1 = torch.tensor(synth.x1(n, 3), dtype=tdt, device="cuda")
    out = torch.empty(ref.numel(), dtype=tdt, device="cuda")
    hd.hd_run(st.h, spec, x1, out)
    torch.cuda.synchronize()
    rel = ((out.double() - ref.double()).norm() / ref.double().norm()).item()
    assert rel <= TOL[dtype], rel
    st.close()


def test_map_options_single_trial_teacher_forced():
    import paper_2101_07464_gb300 as hd
    n = 400_009
    probe = hd.HD("haar", n, n, 6, 1, "f32")
    opts = probe.map_options()
    probe.close()
    assert len(opts) >= 2, opts
    assert opts[0][0] > opts[-1][0] >= 16
    for o in range(len(opts)):
        errs = teacher_forced("haar", n, n, 6, seed=77, dtype="f32", schedule=ALT,
                              setup=lambda g: g.set_tuning([1, o] + [0, 0] * (KINDS * BUCKETS)))
        assert errs.max() <= TOL["f32"], (o, errs)


def test_map_options_batch_of_unequal_trials():
    import paper_2101_07464_gb300 as hd
    ns = [1000, 300_007, 2047, 150_001, 64, 90_001]
    ms = [n // 2 for n in ns]
    T = 10
    flags = [ALT(t) for t in range(1, T + 1)]

    def run(opt):
        b = hd.HDBatch("ginibre", ms, ns, T, 5, "f64")
        b.set_trial_sigmas([m ** -0.5 for m in ms])
        opts = b.map_options()
        if opt >= len(opts):
            b.close()
            return None, opts
        b.set_tuning([1, opt] + [0, 0] * (KINDS * BUCKETS))
        x = torch.tensor(np.concatenate([synth.x1(n, 5, trial=i) for i, n in enumerate(ns)]),
                         dtype=torch.float64, device="cuda")
        out = torch.empty(sum(ns), dtype=torch.float64, device="cuda")
        hd.hd_run(b.h, hd.make_run_spec(flags, "tanh", use_graph=False), x, out)
        torch.cuda.synchronize()
        off = b.off_n.copy()
        b.close()
        return (out.cpu().numpy(), off), opts

    (ref, off), opts = run(0)
    assert len(opts) >= 2, opts
    for o in range(1, len(opts)):
        (got, _), _ = run(o)
        for i in range(len(ns)):
            a, r = got[off[i]:off[i + 1]], ref[off[i]:off[i + 1]]
            assert np.linalg.norm(a - r) <= 1e-12 * np.linalg.norm(r), (o, i)


def test_autotune_cache_and_words():
    import paper_2101_07464_gb300 as hd
    n, T = 250_007, 12
    flags = [ALT(t) for t in range(1, T + 1)]
    spec = hd.make_run_spec(flags, "tanh", use_graph=True)
    x1 = torch.tensor(synth.x1(n, 8), dtype=torch.float64, device="cuda")
    st = hd.HD("haar", n, n, T, 8, "f64")
    assert st.tuning() == [1, 0] + [0, 0] * (KINDS * BUCKETS)
    out0 = torch.empty(n, dtype=torch.float64, device="cuda")
    hd.hd_run(st.h, spec, x1, out0)
    st.autotune(flags, "tanh", x1, reps=1)
    assert st.counts() == (0, 0, 0)
    w = st.tuning()
    assert len(w) == hd.binding.HD_TUNE_WORDS and w[0] == 1 and 0 <= w[1] < len(st.map_options())
    shapes = w[2:]
    assert all(v in (0, 1, 2, 4, 8) for v in shapes)
    assert any(v != 0 for v in shapes)   # the ranges this trajectory visits were measured
    out1 = torch.empty(n, dtype=torch.float64, device="cuda")
    hd.hd_run(st.h, spec, x1, out1)
    torch.cuda.synchronize()
    rel = ((out1 - out0).norm() / out0.norm()).item()
    assert rel <= 1e-12, rel
    # a new state of the same shape starts from the cached choice; another shape does not
    st2 = hd.HD("haar", n, n, T, 99, "f64")
    assert st2.tuning() == w
    st3 = hd.HD("haar", n + 1, n + 1, T, 99, "f64")
    assert st3.tuning() == [1, 0] + [0, 0] * (KINDS * BUCKETS)
    # words round trip, rejection of bad words, reset to the rules
    st3.set_tuning(forcing(4, 2))
    assert st3.tuning() == forcing(4, 2)
    for bad in ([2] + w[1:], [1, 99] + w[2:], forcing(3, 2), forcing(4, 0), w[:10]):
        with pytest.raises(hd.HDError) as ei:
            st3.set_tuning(bad)
        assert ei.value.code == 1
    st3.set_tuning([])
    assert st3.tuning() == [1, 0] + [0, 0] * (KINDS * BUCKETS)
    for s in (st, st2, st3):
        s.close()


def test_autotune_batched_amp():
    import paper_2101_07464_gb300 as hd
    ns = [1200, 40_009, 3001, 20_011]
    ms = [n // 2 for n in ns]
    T = 12
    b = hd.HDBatch("ginibre", ms, ns, T, 4, "f64")
    b.set_trial_sigmas([m ** -0.5 for m in ms])
    beta = np.concatenate([synth.bernoulli_gauss(n, 4, trial=i) for i, n in enumerate(ns)])
    w = np.concatenate([synth.noise(m, 4, trial=i) for i, m in enumerate(ms)])
    bt = torch.tensor(beta, dtype=torch.float64, device="cuda")
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    flags = [ALT(t) for t in range(1, T + 1)]
    spec = hd.make_run_spec(flags, "amp", 1.1, use_graph=True, aux=wt)
    out0 = torch.empty(sum(ns), dtype=torch.float64, device="cuda")
    hd.hd_run(b.h, spec, bt, out0)
    b.autotune(flags, "amp", bt, a=1.1, reps=1, aux=wt)
    out1 = torch.empty(sum(ns), dtype=torch.float64, device="cuda")
    hd.hd_run(b.h, spec, bt, out1)
    torch.cuda.synchronize()
    rel = ((out1 - out0).norm() / out0.norm()).item()
    assert rel <= 1e-9, rel
    b.close()
