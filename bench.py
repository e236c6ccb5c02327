"""Benchmark of the Householder Dice hot path on one GB300 (or N, one process per GPU).

Workload (the paper's method on its Haar ensemble, Algorithm 2): Q ~ Haar(n), n = 10^6,
T = 100 products alternating Q and Q^T, dynamics x_{t+1} = sign(M_t x_t) + 0.5 x_{t-1},
x_1 ~ N(0, I_n) (seeded, synthetic).  One bench "step" is one whole trajectory: T products
(every row of the hot path: draws, the data-side reflector products, the new reflectors,
the outputs) plus the dynamics, all in libhd.so kernels, replayed from one CUDA graph.
Metric: n T^2 / s (the O(nT^2) work unit of the method).  The FP32-storage form is the
headline line; the plain FP64 form is measured on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f32|f64] [--impl reference]

--impl reference times the CPU FP64 oracle on the host cores over the same workload at full
n: whole trajectories when they fit the run's time bound, else the first products of each,
with the whole trajectory's time extrapolated from a fitted per-product cost.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT, T_DEFAULT = 10 ** 6, 100
REFERENCE_TIME_LIMIT_S = 180.0   # bound on a whole --impl reference run (warm-up + timed steps)
METRIC = "HD throughput n*T^2/s (Haar n=1e6, T=100, Q/Q^T alternating)"
UNIT = "n*T^2/s"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--T", type=int, default=T_DEFAULT)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 side measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-amp", action="store_true", help="skip the batched AMP measurement")
    ap.add_argument("--amp-trials", type=int, default=4096)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the reverse-mode measurement")
    ap.add_argument("--no-ista", action="store_true", help="skip the differentiable ISTA workload")
    ap.add_argument("--no-spectral", action="store_true", help="skip the spectral-method workload")
    ap.add_argument("--no-paper-ista", action="store_true",
                    help="skip the paper's timed run (lasso ISTA, Gin(n/2, n), n = 1e7, FP64)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large configuration (Haar n = 2e7, T = 256, forward and reverse mode)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch shapes (no hd_autotune before timing)")
    return ap.parse_args(argv)


def schedule(T):
    return [1 if t % 2 == 0 else 0 for t in range(1, T + 1)]


def parse_args_for_test(argv):
    return parse(argv)


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(secs, dist, device="cuda"):
    """The slowest rank's time (every rank gets it); `dist` is torch.distributed or None."""
    if dist is None:
        return secs
    import torch
    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, secs):
    """Whole-job throughput: every rank processed units_per_rank in at most secs (weak scaling:
    one independent trial per rank, Philox trial word = rank)."""
    return float(units_per_rank) * world / secs


# ----------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
def oracle_sample(n, T, seed, time_limit_s, max_products=None):
    """Run the oracle's first products of the workload until time_limit_s; returns
    (products done, seconds, threads, seconds of each product including its dynamics)."""
    import numpy as np
    import torch
    import synth
    from oracle.dynamics import f_sign_mem
    from oracle.hd import HaarOracle
    ora = HaarOracle(n, T, seed)
    x = synth.x1(n, seed)
    xp = np.zeros(n)
    sched = schedule(T)
    per = []
    t0 = time.perf_counter()
    for t in range(T):
        t1 = time.perf_counter()
        y = ora.apply(x, bool(sched[t])).numpy()
        x, xp = f_sign_mem(y, x, xp), x
        per.append(time.perf_counter() - t1)
        if time.perf_counter() - t0 > time_limit_s or (max_products and len(per) >= max_products):
            break
    return len(per), time.perf_counter() - t0, torch.get_num_threads(), per


def trajectory_seconds(T, samples):
    """Seconds of a whole T-product trajectory from timed samples of its first products.

    samples: lists of per-product seconds, each starting at product 1.  When every sample
    covers all T products this is their mean total.  Otherwise product t costs a fixed part
    (draws, norms, dynamics: O(n)) plus a part that grows with the t - 1 stored reflectors it
    applies (O(n t)), so a least-squares fit of a + b t over all sampled products (a, b >= 0)
    gives the whole trajectory as sum_{t<=T} (a + b t).  Returns (seconds, a, b, exact)."""
    import numpy as np
    if all(len(s) == T for s in samples):
        return float(np.mean([sum(s) for s in samples])), None, None, True
    t = np.concatenate([np.arange(1, len(s) + 1) for s in samples]).astype(np.float64)
    y = np.concatenate([np.asarray(s, dtype=np.float64) for s in samples])
    if len(np.unique(t)) > 1:
        b, a = np.polyfit(t, y, 1)
    else:
        a, b = float(y.mean()), 0.0
    if b < 0.0:
        a, b = float(y.mean()), 0.0
    if a < 0.0:
        a, b = 0.0, float(np.dot(t, y) / np.dot(t, t))
    return float(T * a + b * T * (T + 1) / 2.0), float(a), float(b), False


def oracle_throughput(n, T, samples):
    """n T^2 per second of the whole trajectory, and a description of how it was obtained."""
    secs, a, b, exact = trajectory_seconds(T, samples)
    k = min(len(s) for s in samples)
    if exact:
        how = "all %d of %d products at n=%d, mean of %d run(s)" % (T, T, n, len(samples))
    else:
        how = ("first %d of %d products at n=%d timed (%d run(s)); whole trajectory extrapolated "
               "with product t costing a + b t, a = %.1f ms, b = %.2f ms, fitted to every "
               "sampled product: %.1f s" % (k, T, n, len(samples), a * 1e3, b * 1e3, secs))
    return float(n) * T * T / secs, secs, how


def run_reference(args):
    rank, world, _ = dist_info()
    if world > 1 and rank != 0:
        return
    n, T = args.n, args.T
    # the whole run (warm-up and timed steps) is bounded by about REFERENCE_TIME_LIMIT_S: the
    # first warm-up run sets how many of the T products fit a step's share of it, and every
    # later run times that many
    share = REFERENCE_TIME_LIMIT_S / max(1, args.warmup + args.steps)
    k, _, _, _ = oracle_sample(n, T, args.seed, time_limit_s=share)
    times, samples = [], []
    for i in range(args.warmup + args.steps):
        if i == 0 and args.warmup > 0:
            continue   # the calibration run above is the first warm-up
        done, secs, thr, per = oracle_sample(n, T, args.seed, time_limit_s=1e9, max_products=k)
        if i >= args.warmup:
            times.append(secs)
            samples.append(per)
    value, traj_s, how = oracle_throughput(n, T, samples)
    mean = statistics.mean(times)
    sample = how + " (Haar, Q/Q^T alternating, sign dynamics), FP64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
            "trajectory_s": traj_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "haar_sign n=%d T=%d (%s)" % (
                           n, T, "whole trajectory per step" if k >= T else
                           "per step: first %d products, throughput extrapolated" % k),
                       "n": n, "T": T},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes / algorithmic bytes of one k_update launch (k = 60, n = 10^6, FP32) from an
# ncu --set full capture of the current kernel; reset to None when the kernel changes.
UPDATE_TRAFFIC_RATIO = 250.15 / 252.0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def time_trajectories(st, spec, x1, xout, steps, warmup, dist):
    """Replay the trajectory graph `steps` times between a barrier and CUDA events on the
    launching stream; returns (seconds, max over ranks; kernels launched in the region)."""
    import torch
    import paper_2101_07464_gb300 as hd
    for _ in range(warmup):
        hd.hd_run(st.h, spec, x1, xout)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = hd.hd_get_launches(st.h)
    e0.record(stream)
    for _ in range(steps):
        hd.hd_run(st.h, spec, x1, xout)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = hd.hd_get_launches(st.h) - l0
    secs = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist)
    return secs, launches


def profile_kernels(st, spec, x1, xout, steps):
    """Per-sweep CUDA-event timing of `steps` trajectories (events recorded on the launching
    stream around every sweep, inside the replayed graph; read after each replay)."""
    import torch
    import paper_2101_07464_gb300 as hd
    hd.hd_profile_enable(st.h, True)
    hd.hd_run(st.h, spec, x1, xout)   # re-capture the graph with the event records
    torch.cuda.synchronize()
    hd.hd_profile_read(st.h, clear=True)
    for _ in range(steps):
        hd.hd_run(st.h, spec, x1, xout)
        hd.hd_profile_read(st.h)
    prof = hd.hd_profile_read(st.h)
    hd.hd_profile_enable(st.h, False)
    return prof


def measure_amp_batch(args, rank, world, dist):
    """Batched AMP workload: `amp_trials` independent Gin(m_i, n_i) trials in one state,
    n_i ~ U{1000..100000}, m_i = n_i / 2, entries N(0, 1/m_i), beta ~ Bernoulli(0.1) N(0, 1),
    w ~ N(0, 0.1^2), T = 30 products (Q beta, then Q^T z / Q x alternating), soft threshold
    1.1 ||z|| / sqrt(m), FP32 storage; one hd_run call (one CUDA graph) per trajectory."""
    import numpy as np
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    count, T = args.amp_trials, 30
    ns = synth.batch_sizes(count, 1000, 100000, args.seed + rank)
    ms = ns // 2
    b = hd.HDBatch("ginibre", ms, ns, T, args.seed, "f32", trial=rank * count)
    b.set_trial_sigmas(1.0 / np.sqrt(ms.astype(np.float64)))
    beta = np.concatenate([synth.bernoulli_gauss(int(n), args.seed, trial=i, dtype=np.float32)
                           for i, n in enumerate(ns)])
    w = np.concatenate([synth.noise(int(m), args.seed, trial=i, dtype=np.float32) for i, m in enumerate(ms)])
    bt = torch.from_numpy(beta).cuda()
    wt = torch.from_numpy(w).cuda()
    out = torch.empty_like(bt)
    flags = [t % 2 == 0 for t in range(1, T + 1)]
    spec = hd.make_run_spec(flags, "amp", 1.1, use_graph=True, aux=wt)
    if not args.no_autotune:
        b.autotune(flags, "amp", bt, a=1.1, reps=1, aux=wt)
    for _ in range(2):
        hd.hd_run(b.h, spec, bt, out)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    steps = 3
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        hd.hd_run(b.h, spec, bt, out)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = max_over_ranks(e0.elapsed_time(e1) / 1e3 / steps, dist)
    mse = float(((out.double() - bt.double()) ** 2).sum().item() / float(ns.sum()))
    sum_n, sum_mn = float(ns.sum()), float((ns + ms).sum())
    credited = sum_mn * 4.0 * T * (T + 1) / 2.0
    b.close()
    return {"metric": "trials*n*T^2/s", "value": job_throughput(sum_n * T * T, world, secs),
            "ms_per_trajectory": secs * 1e3, "trials": count * world, "sum_n": sum_n * world, "T": T,
            "dtype": "f32 (FP64 coefficients)", "graph": "one CUDA graph per trajectory",
            "credited_GBps": credited / secs / 1e9, "mse": mse,
            "launch_shapes": "built-in" if args.no_autotune else "hd_autotune (untimed, before the runs)",
            "config": "Gin(m_i, n_i), n_i ~ U{1000..100000}, m_i = n_i/2, AMP soft threshold 1.1 sigma_t"}


def measure_adjoint(args, rank, world, dist):
    """Reverse mode: gradient of <c, x_{T+1}> with respect to x_1 and the per-step parameters
    theta_t of x_{t+1} = tanh(theta_t y_t) + 0.3 x_{t-1} on Haar(n), n = 10^6, T = 100 products
    Q / Q^T alternating, FP32 storage (paper_2101_07464_gb300.autograd.trajectory: forward with
    the library's steps recorded, backward through hd_adjoint_step).  Units n T^2 per
    forward + backward."""
    import numpy as np
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    from paper_2101_07464_gb300.autograd import trajectory
    n, T = 10 ** 6, 100
    sched = [t % 2 == 0 for t in range(1, T + 1)]
    st = hd.HD("haar", n, n, T, args.seed, "f32", trial=rank)
    x1 = torch.tensor(synth.x1(n, args.seed, trial=rank), dtype=torch.float32, device="cuda")
    c = torch.tensor(synth.x1(n, args.seed + 1, trial=rank), dtype=torch.float32, device="cuda")
    theta0 = torch.full((T,), 0.8, dtype=torch.float32, device="cuda")

    def f(t, y, x, xprev, theta):
        v = torch.tanh(theta[t - 1] * y)
        return v if xprev is None else v + 0.3 * xprev

    def one(backward):
        x = x1.clone().requires_grad_(backward)
        th = theta0.clone().requires_grad_(backward)
        out = trajectory(st, x, sched, f, (th,))
        L = torch.dot(c, out)
        if backward:
            L.backward()
        return L

    for _ in range(2):
        one(True)
    torch.cuda.synchronize()
    steps = 3
    t0 = time.perf_counter()
    for _ in range(steps):
        one(True)
    torch.cuda.synchronize()
    fb = (time.perf_counter() - t0) / steps
    t0 = time.perf_counter()
    for _ in range(steps):
        with torch.no_grad():
            one(False)
    torch.cuda.synchronize()
    fw = (time.perf_counter() - t0) / steps
    fb, fw = max_over_ranks(fb, dist), max_over_ranks(fw, dist)
    st.close()
    return {"metric": "n*T^2/s (forward + backward)", "value": job_throughput(float(n) * T * T, world, fb),
            "ms_forward_backward": fb * 1e3, "ms_forward": fw * 1e3, "n": n, "T": T, "dtype": "f32",
            "timing": "wall clock around synchronised whole calls (host-driven steps, torch f_t)",
            "config": "Haar n=1e6, T=100, Q/Q^T alternating, x_{t+1} = tanh(theta_t y_t) + 0.3 x_{t-1}, "
                      "d<c, x_{T+1}>/d(x_1, theta)"}


def measure_ista(args, rank, world, dist):
    """The differentiable ISTA workload: 64 trials of Gin(n, n), n = 2 * 10^5, entries N(0, 1/n),
    50 ISTA iterations x^{k+1} = eta(x^k + tau Q^T (y - Q x^k); theta_k) with y = Q beta* + w
    (101 products: Q beta*, then Q x^k and Q^T r^k alternating), beta* ~ 0.2 delta_0 +
    0.8 N(0, 2^2), w ~ N(0, 0.1^2), FP32 storage; the gradient of (1/n) ||x^50 - beta*||^2 with
    respect to theta_1..theta_50 (0.6) and tau (0.3) through the library's reverse mode.  The
    trials run one after another on one state (Philox trial word per trial); wall clock
    around all of them, synchronised.  Units trials n T^2 per forward + backward, T = 101."""
    import numpy as np
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    from paper_2101_07464_gb300.autograd import trajectory
    n, K, trials = 200_000, 50, 64
    T = 2 * K + 1
    sched = [False] + [bool(t % 2) for t in range(2, T + 1)]
    sigma = n ** -0.5
    st = hd.HD("ginibre", n, n, T, args.seed, "f32", sigma=sigma, trial=rank * trials)

    def make_f(w):
        store = {}

        def f(t, y, x, xprev, theta, tau):
            if t == 1:
                store["y"] = (y + w).detach()
                return torch.zeros_like(y)
            if t % 2 == 0:
                return store["y"] - y
            v = xprev + tau * y
            return torch.sign(v) * torch.clamp(v.abs() - theta[(t - 3) // 2], min=0.0)
        return f

    data = []
    for i in range(trials):
        b = synth.bernoulli_gauss(n, args.seed, trial=rank * trials + i, p_nonzero=0.8, scale=2.0,
                                  dtype=np.float32)
        w = synth.noise(n, args.seed, trial=rank * trials + i, sigma=0.1, dtype=np.float32)
        data.append((torch.from_numpy(b).cuda(), torch.from_numpy(w).cuda()))

    def one(i):
        st.reset()   # the trial word changes only on a reset state
        hd.hd_set_options(st.h, sigma, rank * trials + i, st.stream)
        bt, wt = data[i]
        th = torch.full((K,), 0.6, dtype=torch.float32, device="cuda", requires_grad=True)
        ta = torch.tensor(0.3, dtype=torch.float32, device="cuda", requires_grad=True)
        xK = trajectory(st, bt, sched, make_f(wt), (th, ta))
        L = torch.sum((xK - bt) ** 2) / n
        L.backward()
        return L.detach(), th.grad.norm(), ta.grad.detach()

    one(0)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    res = [one(i) for i in range(trials)]
    torch.cuda.synchronize()
    secs = max_over_ranks(time.perf_counter() - t0, dist)
    st.close()
    mse = float(torch.stack([r[0] for r in res]).mean().item())
    gth = float(torch.stack([r[1] for r in res]).mean().item())
    return {"metric": "trials*n*T^2/s (forward + backward)",
            "value": job_throughput(float(trials) * n * T * T, world, secs),
            "ms_per_trial": secs / trials * 1e3, "trials": trials * world, "n": n, "T": T, "dtype": "f32",
            "mean_loss": mse, "mean_grad_theta_norm": gth,
            "timing": "wall clock around the 64 trials (host-driven steps, torch f_t), synchronised",
            "config": "Gin(n, n), n=2e5, ISTA 50 iterations (101 products), tau=0.3, theta_k=0.6, "
                      "d MSE / d(theta_1..theta_50, tau)"}


def measure_paper_ista(args, rank, world, dist):
    """The one run the paper times (Section 2.1): ISTA for the lasso on Gin(m, n), n = 10^7,
    m = n/2, entries N(0, 1/m), 50 iterations (101 products: Q beta*, then Q x^k and Q^T r^k
    alternating), FP64 like the paper's Julia run.  beta* ~ 0.2 delta_0 + 0.8 N(0, 2^2),
    w ~ N(0, 0.1^2), tau = 0.3, threshold 0.6.  Host-driven products through hd_apply with the
    ISTA update in torch; wall clock around the whole synchronised run, allocation excluded.
    The paper reports 92 s on its CPU machine (context only: other hardware and software)."""
    import numpy as np
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    n, K = 10 ** 7, 50
    m = n // 2
    T = 2 * K + 1
    free, _ = torch.cuda.mem_get_info()
    if free < 40e9:
        return {"skipped": "needs about 40 GB of free device memory, %.0f GB free" % (free / 1e9)}
    st = hd.HD("ginibre", m, n, T, args.seed, "f64", sigma=m ** -0.5, trial=rank)
    beta = torch.tensor(synth.bernoulli_gauss(n, args.seed, trial=rank, p_nonzero=0.8, scale=2.0),
                        dtype=torch.float64, device="cuda")
    w = torch.tensor(synth.noise(m, args.seed, trial=rank, sigma=0.1), dtype=torch.float64, device="cuda")

    def run():
        st.reset()
        y = st.apply(beta, False) + w                 # y = Q beta* + w
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        for _ in range(K):
            r = y - st.apply(x, False)                # y - Q x^k
            v = x + 0.3 * st.apply(r, True)           # x^k + tau Q^T r^k
            x = torch.sign(v) * torch.clamp(v.abs() - 0.6, min=0.0)
        return x

    run()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    x = run()
    torch.cuda.synchronize()
    secs = max_over_ranks(time.perf_counter() - t0, dist)
    mse = float(torch.sum((x - beta) ** 2).item() / n)
    st.close()
    return {"seconds": secs, "paper_seconds": 92.0, "n": n, "m": m, "iterations": K, "products": T,
            "dtype": "f64", "mse": mse,
            "value": job_throughput(float(n) * T * T, world, secs), "unit": UNIT,
            "config": "lasso ISTA on Gin(n/2, n), n=1e7, entries N(0, 1/m), 50 iterations, tau=0.3, "
                      "threshold 0.6, beta* ~ 0.2 delta_0 + 0.8 N(0, 4), w ~ N(0, 0.01)",
            "timing": "wall clock around one synchronised run (host-driven products, torch ISTA update)",
            "note": "the paper's 92 s is a CPU run (Julia, 32 GB machine): context, not a target"}


def measure_spectral(args, rank, world, dist):
    """The spectral method of Section 2.2: A = [I_n 0] Q, Q ~ Haar(m), n = 10^5, m = 2n,
    y = tanh(|A^T xi|), leading eigenvector of D = (1/m) A diag(y) A^T by 100 power iterations
    (201 products: Q^T [xi; 0], then Q^T and Q per iteration), FP64, host-driven products with
    the caller's elementwise steps in torch; wall clock around one synchronised run.  The paper
    reports under 4 s for one extremal eigenpair at n = 10^5 with Krylov-Schur on its CPU
    machine (context only)."""
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    n, K = 10 ** 5, 100
    m = 2 * n
    T = 1 + 2 * K
    st = hd.HD("haar", m, m, T, args.seed, "f64", trial=rank)
    xi = torch.tensor(synth.x1(n, args.seed, trial=rank), dtype=torch.float64, device="cuda")
    x0 = torch.tensor(synth.x1(n, args.seed + 1, trial=rank), dtype=torch.float64, device="cuda")
    z = torch.zeros(m - n, dtype=torch.float64, device="cuda")

    def run():
        st.reset()
        y = torch.tanh(torch.abs(st.apply(torch.cat([xi, z]), True)))
        x = x0 / torch.linalg.vector_norm(x0)
        for _ in range(K):
            v = st.apply(y * st.apply(torch.cat([x, z]), True), False)[:n] / m
            x = v / torch.linalg.vector_norm(v)
        return x

    run()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    x = run()
    torch.cuda.synchronize()
    secs = max_over_ranks(time.perf_counter() - t0, dist)
    rho = float((torch.dot(xi, x) ** 2 / (torch.dot(xi, xi) * torch.dot(x, x))).item())
    st.close()
    return {"seconds": secs, "paper_seconds": 4.0, "n": n, "m": m, "iterations": K, "products": T,
            "dtype": "f64", "rho": rho, "unit": UNIT,
            "value": job_throughput(float(m) * T * T, world, secs),
            "config": "subsampled Haar A = [I 0] Q, Q ~ Haar(2n), n=1e5, y = tanh(|A^T xi|), "
                      "100 power iterations on D = A diag(y) A^T / m",
            "timing": "wall clock around one synchronised run (host-driven products)",
            "note": "the paper's 4 s (Krylov-Schur, CPU, Julia) is context, not a target"}


def measure_large(args, rank, world, dist):
    """The large single-trial configuration: Haar(n), n = 2 * 10^7, T = 256 products, all Q,
    x_{t+1} = normalize(tanh(y_t) + 0.1 x_t), FP32 stacks (2 x 20.5 GB).  Forward: one hd_run
    graph per trajectory (built-in shapes), CUDA events, plus a second pass with events around
    every sweep for the update sweep's algorithmic GB/s.  Reverse mode: d<x_{T+1}, x_1>/d(x_1,
    a_1..a_T) (a_t the per-step mixing, 0.1) through autograd.trajectory with segments of 32
    steps recomputed by hd_probe, wall clock around one whole synchronised call."""
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    from paper_2101_07464_gb300.autograd import trajectory
    n, T, seg = 2 * 10 ** 7, 256, 32
    free, _ = torch.cuda.mem_get_info()
    if free < 120e9:
        return {"skipped": "needs about 120 GB of free device memory, %.0f GB free" % (free / 1e9)}
    flags = [False] * T
    st = hd.HD("haar", n, n, T, args.seed, "f32", trial=rank)
    x1 = torch.tensor(synth.x1(n, args.seed, trial=rank), dtype=torch.float32, device="cuda")
    x1 = x1 / x1.norm()
    out = torch.empty_like(x1)
    spec = hd.make_run_spec(flags, "norm_tanh", 0.1, use_graph=True)
    hd.hd_run(st.h, spec, x1, out)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hd.hd_run(st.h, spec, x1, out)
    e1.record(stream)
    torch.cuda.synchronize()
    fw = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist)
    prof = profile_kernels(st, spec, x1, out, 1)
    peak, _ = measured_peaks()
    per = {k: (v[2] / (v[0] / 1e3) / 1e9 if v[0] else None) for k, v in prof.items()}

    def f(t, y, x, xprev, a):
        v = torch.tanh(y) + a[t - 1] * x
        return v / torch.sqrt(torch.sum(v.double() * v.double())).to(v.dtype)

    a = torch.full((T,), 0.1, dtype=torch.float32, device="cuda", requires_grad=True)
    xg = x1.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xo = trajectory(st, xg, flags, f, (a,), checkpoint=seg)
    L = torch.dot(xo, x1)
    L.backward()
    torch.cuda.synchronize()
    fb = max_over_ranks(time.perf_counter() - t0, dist)
    st.close()
    units = float(n) * T * T
    return {"config": "Haar n=2e7, T=256, all Q, x_{t+1} = normalize(tanh(y_t) + 0.1 x_t), FP32 stacks",
            "forward": {"ms": fw * 1e3, "value": job_throughput(units, world, fw), "unit": UNIT,
                        "update_GBps": per["update"], "update_frac": (per["update"] / peak) if per["update"] else None,
                        "output_GBps": per["output"], "dots_GBps": per["dots"],
                        "launch_shapes": "built-in", "timing": "CUDA events, one graph replay after one warm-up"},
            "adjoint": {"ms_forward_backward": fb * 1e3, "value": job_throughput(units, world, fb), "unit": UNIT,
                        "checkpoint_segment": seg, "loss": "<x_{T+1}, x_1>",
                        "timing": "wall clock around one synchronised forward + backward"}}


def run_ours(args):
    import numpy as np
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    from paper_2101_07464_gb300 import build as hdbuild

    rank, world, local = dist_info()
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    torch.cuda.set_device(local)
    hdbuild.build()
    n, T = args.n, args.T
    flags = schedule(T)

    def measure(dtype, profile):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        st = hd.HD("haar", n, n, T, args.seed, dtype, trial=rank)
        spec = hd.make_run_spec(flags, "sign_mem", 0.5, use_graph=True)
        x1 = torch.tensor(synth.x1(n, args.seed, trial=rank), dtype=tdt, device="cuda")
        xout = torch.empty(n, dtype=tdt, device="cuda")
        if not args.no_autotune:   # measured launch shapes, before the timed region
            st.autotune(flags, "sign_mem", x1, a=0.5, reps=2)
        secs, launches = time_trajectories(st, spec, x1, xout, args.steps, args.warmup, dist)
        prof = profile_kernels(st, spec, x1, xout, args.steps) if profile else None
        return st, spec, secs, prof, launches

    clocks = ClockSampler(local)
    clocks.start()
    st, spec, secs, prof, launches = measure(args.dtype, profile=True)
    clk = clocks.stop()
    per_step = secs / args.steps
    units = float(n) * T * T * world
    value = job_throughput(float(n) * T * T, world, per_step)

    # end to end through the public API: pinned host x_1 in, x_{T+1} back, every step
    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    x1h = torch.tensor(synth.x1(n, args.seed, trial=rank), dtype=tdt).pin_memory()
    xouth = torch.empty(n, dtype=tdt).pin_memory()
    for _ in range(args.warmup):
        hd.hd_run(st.h, spec, x1h, xouth)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hd.hd_run(st.h, spec, x1h, xouth)
        torch.cuda.current_stream().synchronize()   # the result is on the host
        float(xouth[0])
    e2e_secs = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = {"value": units / (e2e_secs / args.steps), "unit": UNIT,
           "h2d_bytes_per_step": n * x1h.element_size(), "d2h_bytes_per_step": n * xouth.element_size()}
    st.close()

    # roofline of the dominant kernel (largest total time inside the timed region)
    peak, peak_kind = measured_peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    ms, nl, by = prof[dom]
    achieved = (by / nl) / ((ms / nl) / 1e3) / 1e9 if nl else 0.0
    roofline = {"bound": "hbm", "kernel": {"dots": "k_dots", "update": "k_update",
                                            "output": "k_out_haar"}[dom],
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind,
                "traffic": ((by / nl) * UPDATE_TRAFFIC_RATIO
                            if (nl and dom == "update" and UPDATE_TRAFFIC_RATIO) else None),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_update "
                                  "launch at k = 60 (250.15 MB for 252.0 MB algorithmic), scaled to "
                                  "the average launch by algorithmic bytes",
                "timing": "CUDA events on the launching stream around every sweep, recorded "
                          "in a second pass of the same trajectories (events inside the graph "
                          "would perturb the headline timing)",
                "per_kernel": {k: {"ms_total": v[0], "launches": v[1],
                                   "GBps": (v[2] / (v[0] / 1e3) / 1e9) if v[0] else None}
                               for k, v in prof.items()}}
    if args.dtype == "f64":
        roofline["note"] = "FP64 sweeps are bound by the FP64 FMA rate, not HBM"
    credited = 2.0 * n * tdt.itemsize * T * (T + 1) / 2.0 * world
    step_gbps = credited / per_step / 1e9

    fp64 = None
    if args.dtype == "f32" and not args.no_fp64:
        st64, _, secs64, _, _ = measure("f64", profile=False)
        st64.close()
        fp64 = {"value": units / (secs64 / args.steps), "ms_per_step": secs64 / args.steps * 1e3,
                "unit": UNIT}

    amp = None
    if not args.no_amp:
        amp = measure_amp_batch(args, rank, world, dist)
    adj = None
    if not args.no_adjoint:
        adj = measure_adjoint(args, rank, world, dist)
    ista = None
    if not args.no_ista:
        try:
            ista = measure_ista(args, rank, world, dist)
        except Exception as exc:   # reported in the line, the headline stands
            ista = {"error": "%s: %s" % (type(exc).__name__, exc)}
    paper_ista = None
    if not args.no_paper_ista:
        try:
            paper_ista = measure_paper_ista(args, rank, world, dist)
        except Exception as exc:   # reported in the line, the headline stands
            paper_ista = {"error": "%s: %s" % (type(exc).__name__, exc)}
    spectral = None
    if not args.no_spectral:
        try:
            spectral = measure_spectral(args, rank, world, dist)
        except Exception as exc:   # reported in the line, the headline stands
            spectral = {"error": "%s: %s" % (type(exc).__name__, exc)}
    large = None
    if not args.no_large:
        try:
            large = measure_large(args, rank, world, dist)
        except Exception as exc:   # reported in the line, the headline stands
            large = {"error": "%s: %s" % (type(exc).__name__, exc)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:   # N = 1 only: the oracle is a single-host baseline
        done, csecs, thr, per = oracle_sample(n, T, args.seed, time_limit_s=15.0)
        cval, _, how = oracle_throughput(n, T, [per])
        cpu = {"value": cval, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": "%s, FP64, wall %.1f s" % (how, csecs)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": "haar_sign", "ensemble": "haar", "n": n, "T": T,
                           "schedule": "Q/Q^T alternating", "dynamics": "sign(y)+0.5x_{t-1}",
                           "storage": "FP32 stacks, FP64 coefficients" if args.dtype == "f32"
                           else "FP64", "per_rank": "independent trial (Philox trial word = rank)",
                           "l2": "inputs larger than L2 (two reflector stacks of %.0f MB each)"
                           % (n * T * tdt.itemsize / 1e6),
                           "graph": "one CUDA graph per trajectory",
                           "launch_shapes": "built-in" if args.no_autotune
                           else "hd_autotune (untimed, before the timed region)"},
                "roofline": roofline,
                "step_credited_GBps": step_gbps,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "fp64": fp64, "batched_amp": amp, "adjoint": adj, "ista": ista, "paper_ista": paper_ista, "spectral": spectral, "large": large}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
