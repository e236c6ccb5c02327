"""hd_run (whole trajectory with a built-in dynamics, optionally one CUDA graph) gives the
same trajectory as hd_apply driven step by step with the same dynamics, bit for bit."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _manual(ens, m, n, T, seed, dtype, flags, dyn, a, sigma):
    from paper_2101_07464_gb300 import HD
    tdt = torch.float64 if dtype == "f64" else torch.float32
    st = HD(ens, m, n, T, seed, dtype, sigma=sigma)
    x = torch.tensor(synth.x1(m if flags[0] else n, seed), dtype=tdt, device="cuda")
    xp = torch.zeros(max(m, n), dtype=tdt, device="cuda")
    for t in range(T):
        y = st.apply(x, bool(flags[t]))
        if dyn == "tanh":
            xn = torch.tanh(y)
        elif dyn == "sign_mem":
            xn = torch.sign(y) + a * xp[:y.numel()]
        else:
            v = torch.tanh(y) + a * x
            xn = v / torch.sqrt(torch.sum(v.double() * v.double())).to(tdt)
        xp = torch.zeros(max(m, n), dtype=tdt, device="cuda")
        xp[:x.numel()] = x
        x = xn
    st.close()
    return x


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("ens,m,n,dyn,a,pattern", [
    ("haar", 10007, 10007, "sign_mem", 0.5, "alt"),
    ("haar", 4099, 4099, "norm_tanh", 0.1, "allq"),
    ("ginibre", 3001, 3001, "tanh", 0.0, "allq"),
    ("ginibre", 2001, 5003, "tanh", 0.0, "alt")])
def test_run_matches_apply(dtype, graph, ens, m, n, dyn, a, pattern):
    """The unfused trajectory path: bit for bit the same kernels as hd_apply."""
    import paper_2101_07464_gb300 as hd
    T = 16
    flags = [(t % 2 == 0) if pattern == "alt" else False for t in range(1, T + 1)]
    sigma = 1.0 if ens == "haar" else m ** -0.5
    ref = _manual(ens, m, n, T, 5, dtype, flags, dyn, a, sigma)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    st = hd.HD(ens, m, n, T, 5, dtype, sigma=sigma)
    hd.hd_set_engine(st.h, no_fuse=True)
    spec = hd.make_run_spec(flags, dyn, a, use_graph=graph)
    x1 = torch.tensor(synth.x1(m if flags[0] else n, 5), dtype=tdt, device="cuda")
    out = torch.empty(ref.numel(), dtype=tdt, device="cuda")
    for rep in range(2):   # second call replays the cached graph
        hd.hd_run(st.h, spec, x1, out)
        torch.cuda.synchronize()
        if dyn == "norm_tanh":   # norm reduction order differs from torch's
            rel = ((out.double() - ref.double()).norm() / ref.double().norm()).item()
            assert rel <= (1e-5 if dtype == "f32" else 1e-12), rel
        else:
            assert torch.equal(out, ref), (out - ref).abs().max().item()
    assert st.counts()[0] == T
    st.close()


def test_run_host_buffers_and_dim_check():
    import paper_2101_07464_gb300 as hd
    n, T = 5000, 8
    flags = [t % 2 == 0 for t in range(1, T + 1)]
    st = hd.HD("haar", n, n, T, 9, "f32")
    spec = hd.make_run_spec(flags, "sign_mem", 0.5, use_graph=True)
    x1d = torch.tensor(synth.x1(n, 9), dtype=torch.float32, device="cuda")
    outd = torch.empty(n, dtype=torch.float32, device="cuda")
    hd.hd_run(st.h, spec, x1d, outd)
    x1h = x1d.cpu().pin_memory()
    outh = torch.empty(n, dtype=torch.float32).pin_memory()
    hd.hd_run(st.h, spec, x1h, outh)
    torch.cuda.synchronize()
    assert torch.equal(outh, outd.cpu())
    st.close()
    g = hd.HD("ginibre", 300, 500, 4, 1, "f64", sigma=0.05)
    bad = hd.make_run_spec([False, False, True, True], "tanh")   # Q then Q: 300 != 500
    with pytest.raises(hd.HDError) as ei:
        hd.hd_run(g.h, bad, torch.zeros(500, dtype=torch.float64, device="cuda"),
                  torch.zeros(500, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 2
    g.close()


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("ens,m,n,dyn,a,dtype", [
    ("haar", 10007, 10007, "sign_mem", 0.5, "f64"),
    ("haar", 65_536, 65_536, "tanh", 0.0, "f32"),
    ("haar", 4099, 4099, "tanh", 0.0, "f64"),
    ("ginibre", 2001, 5003, "tanh", 0.0, "f64"),
    ("ginibre", 30_011, 20_011, "tanh", 0.0, "f32"),
    ("ginibre", 3001, 3001, "sign_mem", 0.5, "f64")])
def test_fused_run_matches_apply(graph, ens, m, n, dyn, a, dtype):
    """Q / Q^T alternating with an elementwise f_t: the output sweep of every step but the last
    applies f_t and forms the next step's dot sweep.  The products are the same up to the
    summation order of the dots (FP64 to 1e-12, FP32 to 1e-5 relative)."""
    import paper_2101_07464_gb300 as hd
    T = 16
    flags = [t % 2 == 0 for t in range(1, T + 1)]
    sigma = 1.0 if ens == "haar" else m ** -0.5
    ref = _manual(ens, m, n, T, 7, dtype, flags, dyn, a, sigma)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    st = hd.HD(ens, m, n, T, 7, dtype, sigma=sigma)
    spec = hd.make_run_spec(flags, dyn, a, use_graph=graph)
    x1 = torch.tensor(synth.x1(m if flags[0] else n, 7), dtype=tdt, device="cuda")
    out = torch.empty(ref.numel(), dtype=tdt, device="cuda")
    l0 = hd.hd_get_launches(st.h)
    for rep in range(2):
        hd.hd_run(st.h, spec, x1, out)
        torch.cuda.synchronize()
        rel = ((out.double() - ref.double()).norm() / ref.double().norm()).item()
        assert rel <= (1e-12 if dtype == "f64" else 1e-5), rel
    # two first-draw kernels, then two sweeps per step (the dot sweep of steps 2..T is done by
    # the previous output sweep; step 1 has none) and one dynamics kernel after the last step
    per_run = (hd.hd_get_launches(st.h) - l0) // 2
    assert per_run == 2 + 2 * T + 1, per_run
    st.close()


@pytest.mark.parametrize("ens,dtype", [("haar", "f64"), ("ginibre", "f64"), ("ginibre", "f32")])
def test_back_to_back_products_match_oracle(ens, dtype):
    """Products issued directly one after another on the stream, no kernel or host wait in
    between, at a size with one CTA per sweep (so the next product's sweeps could start on
    idle SMs while the previous one finishes).  The inputs are fixed seeded vectors, so each
    output is compared with the oracle's at the same step."""
    from oracle.hd import make_oracle
    from paper_2101_07464_gb300 import HD
    from gpu_util import TOL
    n, T, seed = 300, 12, 4
    sched = [(t % 2 == 0) or (t % 5 == 0) for t in range(1, T + 1)]
    sigma = 1.0 if ens == "haar" else n ** -0.5
    tdt = torch.float64 if dtype == "f64" else torch.float32
    xs = [synth.x1(n, seed, trial=t) for t in range(T)]
    if dtype == "f32":
        xs = [x.astype(np.float32).astype(np.float64) for x in xs]
    xd = [torch.tensor(x, dtype=tdt, device="cuda") for x in xs]
    ys = [torch.empty(n, dtype=tdt, device="cuda") for _ in range(T)]
    st = HD(ens, n, n, T, seed, dtype, sigma=sigma)
    torch.cuda.synchronize()
    import paper_2101_07464_gb300 as hd
    for t in range(T):
        hd.hd_apply(st.h, xd[t], sched[t], ys[t])
    torch.cuda.synchronize()
    ora = make_oracle(ens, n, n, T, seed, sigma=sigma)
    for t in range(T):
        yo = ora.apply(xs[t], sched[t]).numpy()
        err = np.linalg.norm(ys[t].double().cpu().numpy() - yo) / np.linalg.norm(yo)
        assert err <= TOL[dtype], (t, err)
    st.close()
