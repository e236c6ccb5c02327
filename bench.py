"""Benchmark of the Householder Dice hot path on one GB300 (or N, one process per GPU).

Workload (the paper's method on its Haar ensemble, Algorithm 2): Q ~ Haar(n), n = 10^6,
T = 100 products alternating Q and Q^T, dynamics x_{t+1} = sign(M_t x_t) + 0.5 x_{t-1},
x_1 ~ N(0, I_n) (seeded, synthetic).  One bench "step" is one whole trajectory: T products
(every row of the hot path: draws, the data-side reflector products, the new reflectors,
the outputs) plus the dynamics, all in libhd.so kernels, replayed from one CUDA graph.
Metric: n T^2 / s (the O(nT^2) work unit of the method).  The headline line is the FP64
form (the paper's precision); the FP32-storage form of the same workload is reported beside
it under "fp32" with its own roofline, and the other workloads under their own keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f64|f32] [--impl reference]

Accuracy: every result carries its error against the FP64 oracle (per-step teacher-forced
error, free-running trajectory error, orthogonality defect ||Q^T Q x - x|| / ||x|| per T, or
gradient error).  The oracle runs only in the CPU-baseline leg (cpu_baseline_leg), which
times it for the baseline and computes the reference values these fields compare against.

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
    ap.add_argument("--dtype", default="f64", choices=["f32", "f64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--T", type=int, default=T_DEFAULT)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-side", action="store_true",
                    help="skip the other-precision form of the headline workload")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy fields (and the oracle reference values they need)")
    ap.add_argument("--no-c1", action="store_true", help="skip the small Ginibre configuration")
    ap.add_argument("--no-complex", action="store_true", help="skip the complex (unitary) workload")
    ap.add_argument("--no-fig1a", action="store_true", help="skip the Fig. 1a run (10^5 lasso ISTA trials)")
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
    ap.add_argument("--step-kernel", action="store_true",
                    help="time the headline with the step kernel (one launch per step, hd_set_engine)")
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


# DRAM bytes / algorithmic bytes of one launch of the dominant kernel, from an ncu capture of
# the current kernel at k = 60, n = 10^6; None until a capture of the current kernel exists.
# (FP32: 250.60 MB for 252.0 MB at k = 60; FP64: 494.20 MB for 504.0 MB at k = 60.)
TRAFFIC_RATIO = {"f32": 250.60 / 252.0, "f64": 494.20 / 504.0}
TRAFFIC_KERNEL = "update"
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_update launch "
                  "(k = 60, n = 10^6, same dtype), scaled to the average "
                  "launch by algorithmic bytes")

# Algorithmic FP64 flops per stack element of each sweep in the fused Q / Q^T alternating
# trajectory (2 per FMA): the update sweep forms p = Delta (x - V w) and the two column
# products V^T p~ and V^T g_{t+1}; the fused output sweep forms y = c - V w' and the next
# step's V^T x_{t+1}; the dot sweep V^T x.
# The step kernel runs both sweeps of a step in one launch.
FLOPS_PER_ELEMENT = {"dots": 2.0, "update": 6.0, "output": 4.0, "step": 10.0}
KERNEL_NAME = {"dots": "k_dots", "update": "k_update", "output": "k_out_haar", "step": "k_step"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def fp64_peak():
    """The FP64 FMA pipe rate of this GPU, measured now (hd_fp64_fma_rate), TFLOP/s."""
    import paper_2101_07464_gb300 as hd
    return hd.hd_fp64_fma_rate(iters=1 << 14, reps=5)


def haar_columns(T, step_launches):
    """Columns each kernel kind streams over one Haar trajectory of T products: before step t
    both stacks hold t - 1 reflectors.  The step kernel runs steps 1 .. s (s = step_launches
    per trajectory, 0 or T - 1); the other steps launch one update and one output sweep."""
    s = step_launches
    k_step = float(s * (s - 1) / 2)
    k_rest = float(T * (T - 1) / 2) - k_step
    return {"step": k_step, "update": k_rest, "output": k_rest, "dots": 0.0}


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


def time_engine_ab(st, spec, x1, out, reps):
    """ms per trajectory of hd_run with the two-launch steps and with the step kernel
    (hd_set_engine), CUDA events on the launching stream; the state is left on two launches."""
    import torch
    import paper_2101_07464_gb300 as hd
    res = {}
    stream = torch.cuda.current_stream()
    for name, on in (("two_launches_ms", False), ("step_kernel_ms", True)):
        hd.hd_set_engine(st.h, step_kernel=on)
        for _ in range(2):
            hd.hd_run(st.h, spec, x1, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            hd.hd_run(st.h, spec, x1, out)
        e1.record(stream)
        torch.cuda.synchronize()
        hd.hd_sync(st.h)
        res[name] = e0.elapsed_time(e1) / reps
    hd.hd_set_engine(st.h, step_kernel=False)
    return res


def measure_step_kernel(args, rank):
    """The step kernel (update sweep and fused output sweep in one cooperative launch per
    step) against the default two launches per step, on the Haar workload (n = 10^6, T = 100,
    alternating, sign with memory) in FP64 and FP32 with the built-in launch shapes: ms per
    trajectory, one graph per trajectory, CUDA events."""
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    n, T = args.n, args.T
    flags = schedule(T)
    out = {}
    for dtype in ("f64", "f32"):
        st = hd.HD("haar", n, n, T, args.seed, dtype, trial=rank)
        x1 = torch.tensor(synth.x1(n, args.seed, trial=rank), dtype=st.torch_dtype, device="cuda")
        xo = torch.empty_like(x1)
        spec = hd.make_run_spec(flags, "sign_mem", 0.5, use_graph=True)
        out[dtype] = time_engine_ab(st, spec, x1, xo, 5 if dtype == "f64" else 10)
        st.close()
    out["launch_shapes"] = "built-in"
    out["kernel"] = "k_step (cooperative launch; per-trial release flags between the two sweeps)"
    return out


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
    ab = time_engine_ab(b, spec, bt, out, steps)   # the same trajectory with the step kernel
    sum_n, sum_mn = float(ns.sum()), float((ns + ms).sum())
    credited = sum_mn * 4.0 * T * (T + 1) / 2.0
    b.close()
    return {"metric": "trials*n*T^2/s", "value": job_throughput(sum_n * T * T, world, secs),
            "ms_per_trajectory": secs * 1e3, "trials": count * world, "sum_n": sum_n * world, "T": T,
            "dtype": "f32 (FP64 coefficients)", "graph": "one CUDA graph per trajectory",
            "credited_GBps": credited / secs / 1e9, "mse": mse, "engine_ab": ab,
            "launch_shapes": "built-in" if args.no_autotune else "hd_autotune (untimed, before the runs)",
            "config": "Gin(m_i, n_i), n_i ~ U{1000..100000}, m_i = n_i/2, AMP soft threshold 1.1 sigma_t"}


def measure_adjoint(args, rank, world, dist):
    """Reverse mode: gradient of <c, x_{T+1}> with respect to x_1 and the per-step parameters
    theta_t (2.0) of x_{t+1} = tanh(theta_t y_t) + 0.3 x_{t-1} on Haar(n), n = 10^6, T = 100
    products Q / Q^T alternating, FP32 storage (paper_2101_07464_gb300.autograd.trajectory:
    forward with the library's steps recorded, backward through hd_adjoint_step).  Units n T^2
    per forward + backward.  theta = 2 keeps the trajectory well conditioned under the
    alternating schedule: with theta = 0.8 most of x_{t+1} lies in the span the earlier
    reflectors fix, and FP32 rounding of the inputs alone moves the trajectory by 5e-5 at
    step 32 (oracle, n = 20000), against 7e-8 with theta = 2."""
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
    theta0 = torch.full((T,), 2.0, dtype=torch.float32, device="cuda")

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
                      "theta_t = 2, d<c, x_{T+1}>/d(x_1, theta)"}


def measure_ista(args, rank, world, dist):
    """The differentiable ISTA workload: 64 trials of Gin(n, n), n = 2 * 10^5, entries N(0, 1/n),
    50 ISTA iterations x^{k+1} = eta(x^k + tau Q^T (y - Q x^k); theta_k) with y = Q beta* + w
    (101 products: Q beta*, then Q x^k and Q^T r^k alternating), beta* ~ 0.2 delta_0 +
    0.8 N(0, 2^2), w ~ N(0, 0.1^2), FP32 storage; the gradient of the mean over trials of
    (1/n) ||x^50 - beta*||^2 with respect to theta_1..theta_50 (0.6) and tau (0.3) through the
    library's reverse mode.  All 64 trials are one batched state (Philox trial word per trial):
    every forward product and every reverse step is one set of launches for the whole batch,
    with the ISTA update in torch on the packed vectors.  Wall clock around one synchronised
    forward + backward.  Units trials n T^2 per forward + backward, T = 101."""
    import numpy as np
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    from paper_2101_07464_gb300.autograd import trajectory
    n, K, trials = 200_000, 50, 64
    T = 2 * K + 1
    sched = [False] + [bool(t % 2) for t in range(2, T + 1)]
    sigma = n ** -0.5
    b = hd.HDBatch("ginibre", [n] * trials, [n] * trials, T, args.seed, "f32", sigma=sigma, trial=rank * trials)
    beta = np.concatenate([synth.bernoulli_gauss(n, args.seed, trial=rank * trials + i, p_nonzero=0.8, scale=2.0,
                                                 dtype=np.float32) for i in range(trials)])
    w = np.concatenate([synth.noise(n, args.seed, trial=rank * trials + i, sigma=0.1, dtype=np.float32)
                        for i in range(trials)])
    bt = torch.from_numpy(beta).cuda()
    wt = torch.from_numpy(w).cuda()

    def make_f():
        store = {}

        def f(t, y, x, xprev, theta, tau):
            if t == 1:
                store["y"] = (y + wt).detach()
                return torch.zeros_like(y)
            if t % 2 == 0:
                return store["y"] - y
            v = xprev + tau * y
            return torch.sign(v) * torch.clamp(v.abs() - theta[(t - 3) // 2], min=0.0)
        return f

    def one():
        th = torch.full((K,), 0.6, dtype=torch.float32, device="cuda", requires_grad=True)
        ta = torch.tensor(0.3, dtype=torch.float32, device="cuda", requires_grad=True)
        xK = trajectory(b, bt, sched, make_f(), (th, ta))
        L = torch.sum((xK - bt) ** 2) / (n * trials)
        L.backward()
        return L.detach(), th.grad.norm(), ta.grad.detach()

    one()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        res = one()
    torch.cuda.synchronize()
    secs = max_over_ranks((time.perf_counter() - t0) / reps, dist)
    b.close()
    return {"metric": "trials*n*T^2/s (forward + backward)",
            "value": job_throughput(float(trials) * n * T * T, world, secs),
            "ms_per_batch": secs * 1e3, "ms_per_trial": secs / trials * 1e3, "trials": trials * world, "n": n, "T": T,
            "dtype": "f32", "mean_loss": float(res[0].item()), "grad_theta_norm": float(res[1].item()),
            "timing": "wall clock around one synchronised forward + backward of the 64-trial batch, mean of 3",
            "config": "64 trials of Gin(n, n), n=2e5, ISTA 50 iterations (101 products), tau=0.3, theta_k=0.6, "
                      "d MSE / d(theta_1..theta_50, tau), one batched state (batched reverse mode)"}


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


# ----------------------------------------------------------------------------------------
# The CPU-baseline leg: the only place (besides the reference arm) that runs the oracle.  It
# times the oracle on the headline workload (cpu_baseline) and computes the reference values
# of every accuracy field at the sizes below (full size where the oracle finishes in seconds).
N_ACC_FP32 = 200_000          # Haar workload in FP32: teacher-forced at this n
N_ACC_LARGE, T_LARGE = 10_000, 256
N_ACC_GRAD = 10_000           # reverse-mode gradients against the oracle's float64 autograd
T_ACC_ADJ, K_ACC_ISTA = 24, 10    # steps within the converging trajectories' conditioning
N_ACC_ISTA = 20_000           # lasso ISTA, Gin(n/2, n)
N_ACC_SPECTRAL = 3_000
N_ACC_COMPLEX = 20_000
AMP_ACC_TRIALS = 4


def alt(t):
    return t % 2 == 0


# Smallest alpha_t / ||x_t|| (the part of the step input that the revealed reflectors do not
# already fix) at which per-step parity is meaningful: the unit roundoff over the tolerance.
# Below it the new reflector is built from a tail dominated by rounding (reading A13(i)).
COND_MIN = {"f64": 1.1e-16 / 1e-12, "f32": 6.0e-8 / 1e-5}


def unrevealed_fraction(ora, x, transpose):
    """alpha of the data-side reflector the oracle's last product built, over ||x||."""
    import numpy as np
    r = (ora.L if transpose else ora.R)[-1]
    nx = float(np.linalg.norm(np.asarray(x)))
    return float(r.alpha) / nx if nx > 0 else 0.0


def f32_cast(v):
    import numpy as np
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def cpu_baseline_leg(args, n, T, want_accuracy):
    """Returns (cpu_baseline, refs): the oracle timed on the headline trajectory at full n
    (FP64, every product) and the oracle's reference values of the accuracy fields."""
    import numpy as np
    import torch
    import synth
    from oracle.adjoint import trajectory as oracle_grad_trajectory
    from oracle.dynamics import amp_trace, f_norm_tanh, f_sign_mem, f_tanh, run_trace
    from oracle.hd import make_oracle
    refs = {}
    x1 = synth.x1(n, args.seed)
    t0 = time.perf_counter()
    ora = make_oracle("haar", n, n, T, args.seed)
    xs, ys, fs = run_trace(ora, x1, T, f_sign_mem, alt)
    secs = time.perf_counter() - t0
    cpu = {"value": float(n) * T * T / secs, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
           "sample": "all %d of %d products of one trajectory at n=%d (Haar, Q/Q^T alternating, sign "
                     "dynamics), FP64, wall %.1f s" % (T, T, n, secs)}
    refs["headline"] = {"xs": xs, "ys": ys, "fs": fs}
    if not want_accuracy:
        return cpu, refs
    na = min(n, N_ACC_FP32)
    xa = synth.x1(na, args.seed)
    refs["fp32"] = {"n": na,
                    "teacher": run_trace(make_oracle("haar", na, na, T, args.seed), xa, T, f_sign_mem, alt,
                                         cast=f32_cast),
                    "free": run_trace(make_oracle("haar", na, na, T, args.seed), xa, T, f_sign_mem, alt)}
    # small Ginibre configuration, full size
    nc, Tc = 1000, 10
    oc = make_oracle("ginibre", nc, nc, Tc, args.seed, sigma=nc ** -0.5)
    refs["c1"] = run_trace(oc, synth.x1(nc, args.seed), Tc, f_tanh, lambda t: False)
    # batched AMP: the workload's first trials, FP32 inputs
    ns = synth.batch_sizes(args.amp_trials, 1000, 100000, args.seed)[:AMP_ACC_TRIALS]
    amp = []
    for i, nn in enumerate(ns):
        nn = int(nn)
        mm = nn // 2
        beta = f32_cast(synth.bernoulli_gauss(nn, args.seed, trial=i))
        w = f32_cast(synth.noise(mm, args.seed, trial=i))
        oa = make_oracle("ginibre", mm, nn, 30, args.seed, trial=i, sigma=mm ** -0.5)
        amp.append({"n": nn, "m": mm, "beta": beta, "w": w, "trace": amp_trace(oa, beta, w, 30, cast=f32_cast)})
    refs["amp"] = amp
    # large configuration at reduced n, FP32 inputs
    xl = synth.x1(N_ACC_LARGE, args.seed)
    ol = make_oracle("haar", N_ACC_LARGE, N_ACC_LARGE, T_LARGE, args.seed)
    tl = run_trace(ol, f32_cast(xl / np.linalg.norm(xl)), T_LARGE, f_norm_tanh, lambda t: False, cast=f32_cast)
    # alpha_t / ||x_t||: the part of x_t that the revealed reflectors do not already fix
    frac = [float(r.alpha) / float(np.linalg.norm(x)) for r, x in zip(ol.R, tl[0])]
    refs["large"] = {"n": N_ACC_LARGE, "teacher": tl, "unrevealed_fraction": frac}
    # reverse mode: the adjoint workload's gradients at reduced n (oracle float64 autograd)
    refs["adjoint"] = grad_reference(oracle_grad_trajectory, "adjoint", args.seed)
    refs["ista"] = grad_reference(oracle_grad_trajectory, "ista", args.seed)
    # lasso ISTA (the paper's timed run) and the spectral method at reduced n: every product's
    # input, transpose flag and output
    refs["paper_ista"] = lasso_reference(make_oracle, N_ACC_ISTA, args.seed)
    refs["complex"] = complex_reference(N_ACC_COMPLEX, T, args.seed)
    refs["fig1a"] = fig1a_direct_reference(args.seed)
    refs["spectral"] = spectral_reference(make_oracle, N_ACC_SPECTRAL, args.seed)
    return cpu, refs


def adjoint_problem(kind, n, seed):
    """The reduced-size instance of a reverse-mode workload shared by the oracle reference and
    the GPU check: (ensemble, m, n, T, schedule, f, x1, params, c or None, sigma)."""
    import numpy as np
    import synth
    if kind == "adjoint":
        T = T_ACC_ADJ
        sched = [alt(t) for t in range(1, T + 1)]

        def f(t, y, x, xprev, theta):
            import torch
            v = torch.tanh(theta[t - 1] * y)
            return v if xprev is None else v + 0.3 * xprev
        x1 = f32_cast(synth.x1(n, seed))
        c = f32_cast(synth.x1(n, seed + 1))
        return "haar", n, n, T, sched, f, x1, [np.full(T, 2.0)], c, 1.0
    K = K_ACC_ISTA
    T = 2 * K + 1
    sched = [False] + [bool(t % 2) for t in range(2, T + 1)]
    beta = f32_cast(synth.bernoulli_gauss(n, seed, trial=0, p_nonzero=0.8, scale=2.0))
    w = f32_cast(synth.noise(n, seed, trial=0, sigma=0.1))

    def make_f(wt):
        store = {}

        def f(t, y, x, xprev, theta, tau):
            import torch
            if t == 1:
                store["y"] = (y + wt).detach()
                return torch.zeros_like(y)
            if t % 2 == 0:
                return store["y"] - y
            v = xprev + tau * y
            return torch.sign(v) * torch.clamp(v.abs() - theta[(t - 3) // 2], min=0.0)
        return f
    return "ginibre", n, n, T, sched, make_f, beta, [np.full(K, 0.6), np.float64(0.3)], w, n ** -0.5


def grad_reference(oracle_grad_trajectory, kind, seed):
    import numpy as np
    import torch
    n = N_ACC_GRAD
    ens, m, n, T, sched, f, x1, params, extra, sigma = adjoint_problem(kind, n, seed)
    xt = torch.tensor(x1, dtype=torch.float64, requires_grad=True)
    ps = [torch.tensor(p, dtype=torch.float64, requires_grad=True) for p in params]
    if kind == "adjoint":
        out = oracle_grad_trajectory(ens, m, n, T, seed, sched, f, xt, tuple(ps), sigma=sigma)
        L = torch.dot(torch.tensor(extra, dtype=torch.float64), out)
    else:
        fw = f(torch.tensor(extra, dtype=torch.float64))
        out = oracle_grad_trajectory(ens, m, n, T, seed, sched, fw, xt, tuple(ps), sigma=sigma)
        L = torch.sum((out - xt.detach()) ** 2) / n
    L.backward()
    return {"n": n, "T": T, "loss": float(L.item()), "grad_x1": xt.grad.numpy().copy(),
            "grad_params": [p.grad.numpy().copy() for p in ps]}


def lasso_reference(make_oracle, n, seed):
    """The lasso ISTA of the paper's timed run at size n: y = Q beta + w, then
    x^{k+1} = eta(x^k + tau Q^T (y - Q x^k); 0.6), 50 iterations, FP64."""
    import numpy as np
    import synth
    from oracle.dynamics import soft_threshold
    m, K = n // 2, 50
    ora = make_oracle("ginibre", m, n, 2 * K + 1, seed, sigma=m ** -0.5)
    beta = synth.bernoulli_gauss(n, seed, trial=0, p_nonzero=0.8, scale=2.0)
    w = synth.noise(m, seed, trial=0, sigma=0.1)
    ins, trs, outs, frac = [], [], [], []

    def app(v, tr):
        ins.append(v); trs.append(tr)
        o = ora.apply(v, tr).numpy()
        outs.append(o)
        frac.append(unrevealed_fraction(ora, v, tr))
        return o
    y = app(beta, False) + w
    x = np.zeros(n)
    for _ in range(K):
        r = y - app(x, False)
        x = soft_threshold(x + 0.3 * app(r, True), 0.6)
    return {"ensemble": "ginibre", "m": m, "n": n, "sigma": m ** -0.5, "seed": seed, "ins": ins, "trs": trs,
            "outs": outs, "frac": frac}


FIG1A_DIRECT_TRIALS = 300


def fig1a_direct_reference(seed):
    """The direct approach of Fig. 1a (a dense Gin(n/2, n) matrix per trial, oracle/direct.py)
    at n = 1000 over FIG1A_DIRECT_TRIALS trials: per-iteration mean MSE and its standard error."""
    import numpy as np
    from oracle.direct import ginibre
    n, K = FIG1A_N, FIG1A_K
    m = n // 2
    rng = np.random.default_rng([seed, 1234])
    curves = []
    for _ in range(FIG1A_DIRECT_TRIALS):
        beta = (rng.random(n) < 0.8) * 2.0 * rng.standard_normal(n)
        w = 0.1 * rng.standard_normal(m)
        A = ginibre(rng, m, n, m ** -0.5)
        y = A @ beta + w
        x, mse = np.zeros(n), []
        for _ in range(K):
            v = x + 0.3 * (A.T @ (y - A @ x))
            x = np.sign(v) * np.maximum(np.abs(v) - 0.6, 0.0)
            mse.append(float(np.sum((x - beta) ** 2) / n))
        curves.append(mse)
    c = np.array(curves)
    return {"mean": c.mean(axis=0), "se": c.std(axis=0, ddof=1) / np.sqrt(len(curves)), "trials": len(curves)}


def complex_reference(n, T, seed):
    """The complex workload at size n: the oracle's trajectory of the phase map (all Q), with
    every product's input, flag, output and unrevealed fraction."""
    import numpy as np
    import synth
    from oracle.complex_hd import ComplexHaarOracle
    ora = ComplexHaarOracle(n, T, seed)
    x = synth.x1(n, seed) + 1j * synth.x1(n, seed + 7)
    ins, trs, outs, frac = [], [], [], []
    for t in range(1, T + 1):
        ins.append(x); trs.append(False)
        y = ora.apply(x, False).numpy()
        outs.append(y)
        frac.append(unrevealed_fraction(ora, x, False))
        a = np.abs(y)
        x = np.where(a > 0, y / np.where(a > 0, a, 1.0), 0.0)
    return {"n": n, "seed": seed, "ins": ins, "trs": trs, "outs": outs, "frac": frac}


def spectral_reference(make_oracle, n, seed, K=30):
    """Power iterations of the spectral method at size n (m = 2n): every product's input,
    flag and output."""
    import numpy as np
    import synth
    m = 2 * n
    ora = make_oracle("haar", m, m, 1 + 2 * K, seed)
    xi = synth.x1(n, seed)
    x = synth.x1(n, seed + 1)
    z = np.zeros(m - n)
    ins, trs, outs, frac = [], [], [], []

    def app(v, tr):
        ins.append(v); trs.append(tr)
        o = ora.apply(v, tr).numpy()
        outs.append(o)
        frac.append(unrevealed_fraction(ora, v, tr))
        return o
    yv = np.tanh(np.abs(app(np.concatenate([xi, z]), True)))
    x = x / np.linalg.norm(x)
    for _ in range(K):
        v = app(yv * app(np.concatenate([x, z]), True), False)[:n] / m
        x = v / np.linalg.norm(v)
    return {"ensemble": "haar", "m": m, "n": m, "sigma": 1.0, "seed": seed, "ins": ins, "trs": trs, "outs": outs,
            "frac": frac}


# ----------------------------------------------------------------------------------------
# Accuracy fields (GPU side): the library's results against the oracle reference values that
# cpu_baseline_leg computed.  Element-wise errors are max_i |a_i - b_i| / max_i |b_i| per step.
def _g3(v):
    return float("%.3g" % v)


def per_t(errs):
    return {"max": _g3(max(errs)) if errs else None, "per_T": [_g3(e) for e in errs]}


def max_rel_dev(a, b, head=0):
    """Element-wise error of a (CUDA tensor) against the oracle's b (numpy float64): rows below
    `head` (the pivot rows fixed by the reflectors so far, t after step t) relative to
    ||b||_2, the others relative to max_i |b_i|.  The oracle forms each pivot row as the
    difference of two terms of the size of ||x_t|| (eq. Householder applied literally), so
    its own rounding there scales with the norm."""
    import torch
    bt = torch.from_numpy(b).to(device=a.device)
    d = (a.to(bt.dtype) - bt).abs()
    h = min(int(head), bt.numel())
    s = bt.abs().max().item()
    e = (d[h:].max().item() / s if s > 0 else d[h:].max().item()) if h < bt.numel() else 0.0
    if h > 0:
        nb = bt.norm().item()
        e = max(e, d[:h].max().item() / nb if nb > 0 else d[:h].max().item())
    return e


def rows_of(vs, L, tdt):
    import torch
    out = torch.zeros((len(vs), L), dtype=tdt, device="cuda")
    for i, v in enumerate(vs):
        out[i, :v.shape[0]] = torch.from_numpy(v).to(device="cuda", dtype=tdt)
    return out


def run_records(st, flags, dyn, a, x1, L, given=None, aux=None, graph=True):
    """One hd_run of the trajectory with y_t (and f_t's result) recorded, teacher-forced when
    `given` holds the next inputs; returns the two T x L device records."""
    import torch
    import paper_2101_07464_gb300 as hd
    T = len(flags)
    tdt = st.torch_dtype
    yrec = torch.zeros((T, L), dtype=tdt, device="cuda")
    xrec = torch.zeros((T, L), dtype=tdt, device="cuda")
    out = torch.empty(L, dtype=tdt, device="cuda")
    spec = hd.make_run_spec(flags, dyn, a, use_graph=graph, aux=aux, y_record=yrec, x_record=xrec, x_given=given)
    hd.hd_run(st.h, spec, x1, out)
    torch.cuda.synchronize()
    return yrec, xrec


def ortho_defect(st, xs, flags):
    """||Q^T Q x_t - x_t|| / ||x_t|| (Q^T applied to Q x_t, both through hd_probe on the
    state's revealed part) for each recorded input x_t (host float64 vectors)."""
    import torch
    out = []
    for x, tr in zip(xs, flags):
        xt = torch.from_numpy(x).to(device="cuda", dtype=st.torch_dtype)
        y, _ = st.probe(xt, bool(tr))
        back, _ = st.probe(y, not bool(tr))
        out.append(((back.double() - xt.double()).norm() / xt.double().norm()).item())
    return out


def accuracy_haar_sign(dtype, n, T, seed, teacher, free):
    """Teacher-forced and free-running per-step errors and the orthogonality defect of the
    benchmarked trajectory path (hd_run, fused sweeps, one graph) at size n."""
    import torch
    import paper_2101_07464_gb300 as hd
    xs, ys, _ = teacher
    flags = [alt(t) for t in range(1, T + 1)]
    st = hd.HD("haar", n, n, T, seed, dtype)
    tdt = st.torch_dtype
    x1 = torch.from_numpy(xs[0]).to(device="cuda", dtype=tdt)
    yrec, _ = run_records(st, flags, "sign_mem", 0.5, x1, n, given=rows_of(xs[1:] + [xs[-1]], n, tdt))
    tf = [max_rel_dev(yrec[t], ys[t], t + 1) for t in range(T)]
    orth = ortho_defect(st, xs, flags)
    del yrec
    fx, fy, _ = free
    yrec, _ = run_records(st, flags, "sign_mem", 0.5, torch.from_numpy(fx[0]).to(device="cuda", dtype=tdt), n)
    fr = [max_rel_dev(yrec[t], fy[t], t + 1) for t in range(T)]
    st.close()
    return {"n": n, "teacher_forced_error": per_t(tf), "free_run_error": per_t(fr),
            "orthogonality_defect": per_t(orth),
            "how": "per step t: max_i |y_gpu - y_oracle| / max_i |y_oracle| (the t pivot rows relative "
                   "to ||y_oracle||, where the oracle's own rounding scales with the norm); teacher-forced = both "
                   "given the oracle's x_t (hd_run x_given), free-run = each on its own trajectory; "
                   "defect = ||Q^T Q x_t - x_t|| / ||x_t|| by hd_probe on the final state"}


def accuracy_products(ref, dtype):
    """Per-product teacher-forced error of host-driven hd_apply products (the path of the
    host-driven workloads) on the oracle's inputs."""
    import paper_2101_07464_gb300 as hd
    import torch
    st = hd.HD(ref["ensemble"], ref["m"], ref["n"], len(ref["ins"]), ref["seed"], dtype, sigma=ref["sigma"])
    errs = []
    for x, tr, yo in zip(ref["ins"], ref["trs"], ref["outs"]):
        y = st.apply(torch.from_numpy(x).to(device="cuda", dtype=st.torch_dtype), tr)
        errs.append(max_rel_dev(y, yo, len(errs) + 1))
    st.close()
    ok = [e for e, f in zip(errs, ref["frac"]) if f >= COND_MIN[dtype]]
    return {"error": per_t(errs), "unrevealed_fraction": per_t(ref["frac"]),
            "max_error_while_conditioned": _g3(max(ok)) if ok else None, "products_conditioned": len(ok)}


def accuracy_c1(ref, seed):
    """Small Ginibre configuration (full size): teacher-forced and free-running errors of the
    hd_run path (all Q, unfused sweeps, one graph)."""
    import torch
    import paper_2101_07464_gb300 as hd
    xs, ys, fs = ref
    n, T = 1000, len(ys)
    flags = [False] * T
    st = hd.HD("ginibre", n, n, T, seed, "f64", sigma=n ** -0.5)
    x1 = torch.from_numpy(xs[0]).to("cuda")
    yrec, _ = run_records(st, flags, "tanh", 0.0, x1, n, given=rows_of(xs[1:] + [xs[-1]], n, torch.float64))
    tf = [max_rel_dev(yrec[t], ys[t], t + 1) for t in range(T)]
    yrec, _ = run_records(st, flags, "tanh", 0.0, x1, n)
    fr = [max_rel_dev(yrec[t], ys[t], t + 1) for t in range(T)]
    st.close()
    return {"teacher_forced_error": per_t(tf), "free_run_error": per_t(fr)}


def accuracy_amp(ref, seed):
    """Batched AMP (FP32): the workload's first trials in one batched state, teacher-forced
    through the fused AMP sweep; per step the largest error over the trials of the products
    and of the AMP updates."""
    import numpy as np
    import torch
    import paper_2101_07464_gb300 as hd
    ns = [r["n"] for r in ref]
    ms = [r["m"] for r in ref]
    T = 30
    b = hd.HDBatch("ginibre", ms, ns, T, seed, "f32")
    b.set_trial_sigmas([m ** -0.5 for m in ms])
    off_n, off_m = b.off_n, b.off_m
    L = int(max(off_n[-1], off_m[-1]))
    given = torch.zeros((T, L), dtype=torch.float32, device="cuda")
    for t in range(1, T):
        row = np.concatenate([r["trace"]["used"][t - 1] for r in ref])
        given[t - 1, :row.shape[0]] = torch.from_numpy(row).to(device="cuda", dtype=torch.float32)
    beta = torch.from_numpy(np.concatenate([r["beta"] for r in ref])).to(device="cuda", dtype=torch.float32)
    w = torch.from_numpy(np.concatenate([r["w"] for r in ref])).to(device="cuda", dtype=torch.float32)
    yrec, xrec = run_records(b, [alt(t) for t in range(1, T + 1)], "amp", 1.1, beta, L, given=given, aux=w)
    ep, eu = [], []
    for t in range(1, T + 1):
        off = off_n if t % 2 == 0 else off_m
        ep.append(max(max_rel_dev(yrec[t - 1, int(off[i]):int(off[i + 1])], r["trace"]["products"][t - 1], t)
                      for i, r in enumerate(ref)))
        eu.append(max(max_rel_dev(xrec[t - 1, int(off[i]):int(off[i + 1])], r["trace"]["updates"][t - 1], t)
                      for i, r in enumerate(ref)))
    b.close()
    return {"trials_checked": len(ref), "n": ns, "teacher_forced_error": per_t(ep),
            "update_error": per_t(eu),
            "how": "the workload's first %d trials (same sizes, seeds and trial words), FP32, "
                   "teacher-forced AMP vectors (hd_run x_given); products y_t and updates z^k / x^k "
                   "element-wise against the oracle's AMP" % len(ref)}


def accuracy_large(ref, seed):
    """The large configuration's path (all Q, norm-tanh, unfused sweeps, one graph, FP32) at
    reduced n over all T = 256 steps: teacher-forced errors and the orthogonality defect."""
    import torch
    import paper_2101_07464_gb300 as hd
    n = ref["n"]
    xs, ys, _ = ref["teacher"]
    T = len(ys)
    flags = [False] * T
    st = hd.HD("haar", n, n, T, seed, "f32")
    x1 = torch.from_numpy(xs[0]).to(device="cuda", dtype=torch.float32)
    yrec, _ = run_records(st, flags, "norm_tanh", 0.1, x1, n, given=rows_of(xs[1:] + [xs[-1]], n, torch.float32))
    tf = [max_rel_dev(yrec[t], ys[t], t + 1) for t in range(T)]
    orth = ortho_defect(st, xs, flags)
    st.close()
    frac = ref["unrevealed_fraction"]
    ok = [e for e, f in zip(tf, frac) if f >= COND_MIN["f32"]]
    return {"n": n, "T": T, "teacher_forced_error": per_t(tf), "orthogonality_defect": per_t(orth),
            "unrevealed_fraction": per_t(frac),
            "max_error_while_conditioned": _g3(max(ok)) if ok else None,
            "steps_conditioned": len(ok),
            "note": "this dynamics converges: alpha_t / ||x_t|| (the part of x_t the revealed reflectors do "
                    "not fix, from the oracle) falls geometrically, so each new reflector is built from an "
                    "ever smaller tail and FP32 rounding of order 6e-8 ||x_t|| / alpha_t enters it.  Per-step "
                    "parity is meaningful while alpha_t / ||x_t|| >= 6e-3, the FP32 unit roundoff over the "
                    "1e-5 tolerance (max_error_while_conditioned); "
                    "later steps remain valid samples of the ensemble but follow their own rounding"}


def accuracy_grad(kind, ref, seed):
    """Reverse mode at reduced n, in the timed entry's precision (FP32): the gradients against
    the oracle's float64 autograd on the same FP32-representable inputs."""
    import numpy as np
    import torch
    import paper_2101_07464_gb300 as hd
    from paper_2101_07464_gb300.autograd import trajectory
    ens, m, n, T, sched, f, x1, params, extra, sigma = adjoint_problem(kind, ref["n"], seed)
    st = hd.HD(ens, m, n, T, seed, "f32", sigma=sigma)
    xt = torch.from_numpy(x1).to(device="cuda", dtype=torch.float32).requires_grad_(True)
    ps = [torch.tensor(np.asarray(p), dtype=torch.float32, device="cuda").requires_grad_(True) for p in params]
    if kind == "adjoint":
        out = trajectory(st, xt, sched, f, tuple(ps))
        L = torch.dot(torch.from_numpy(extra).to(device="cuda", dtype=torch.float32), out)
    else:
        out = trajectory(st, xt, sched, f(torch.from_numpy(extra).to(device="cuda", dtype=torch.float32)), tuple(ps))
        L = torch.sum((out - xt.detach()) ** 2) / n
    L.backward()
    st.close()

    def rel(a, b):
        a, b = np.atleast_1d(np.asarray(a, dtype=np.float64)), np.atleast_1d(b)
        return _g3(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    res = {"n": n, "T": T, "loss_rel_error": _g3(abs(L.item() - ref["loss"]) / max(abs(ref["loss"]), 1e-300)),
           "grad_params_rel_error": [rel(p.grad.double().cpu().numpy(), g) for p, g in zip(ps, ref["grad_params"])]}
    if kind == "adjoint":
        res["grad_x1_rel_error"] = rel(xt.grad.double().cpu().numpy(), ref["grad_x1"])
    res["how"] = ("FP32 reverse mode (autograd.trajectory) against the oracle's float64 autograd, "
                  "relative 2-norm error of each gradient, at reduced n over the first %d products of the "
                  "adjoint workload and the first %d ISTA iterations: both trajectories converge (the "
                  "oracle's alpha_t / ||x_t|| falls below the FP32 unit roundoff over 1e-5 after about "
                  "20 products), and later FP32 and FP64 trajectories separate by that conditioning, not "
                  "by the reverse mode" % (T_ACC_ADJ, K_ACC_ISTA))
    return res


def accuracy_complex(ref):
    """Complex workload at reduced n, complex FP64, every product teacher-forced."""
    import torch
    import paper_2101_07464_gb300 as hd
    st = hd.HDComplex("haar", ref["n"], ref["n"], len(ref["ins"]), ref["seed"], "f64")
    errs, ndef = [], []
    for x, tr, yo in zip(ref["ins"], ref["trs"], ref["outs"]):
        xt = torch.from_numpy(x).to("cuda")
        y = st.apply(xt, tr)
        errs.append(max_rel_dev(y, yo, len(errs) + 1))
        ndef.append(abs((y.norm() / xt.norm()).item() - 1.0))
    st.close()
    ok = []
    for e, f in zip(errs, ref["frac"]):
        if f < COND_MIN["f64"]:
            break
        ok.append(e)
    return {"n": ref["n"], "teacher_forced_error": per_t(errs), "norm_defect": per_t(ndef),
            "unrevealed_fraction": per_t(ref["frac"]),
            "max_error_while_conditioned": _g3(max(ok)) if ok else None, "steps_conditioned": len(ok),
            "how": "complex FP64, every product teacher-forced on the oracle's inputs (hd_complex_apply); "
                   "norm_defect = | ||y_t|| / ||x_t|| - 1 | (unitarity); parity is meaningful while the "
                   "oracle's alpha_t / ||x_t|| >= 1.1e-4"}


def measure_c1(args):
    """Small Ginibre configuration: Gin(n, n), n = 1000, entries N(0, 1/n), T = 10, all Q,
    x_{t+1} = tanh(y_t), FP64: microseconds per product through hd_run, replayed as one CUDA
    graph and launched stream-ordered without the graph."""
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    n, T = 1000, 10
    flags = [False] * T
    st = hd.HD("ginibre", n, n, T, args.seed, "f64", sigma=n ** -0.5)
    x1 = torch.tensor(synth.x1(n, args.seed), dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    res = {}
    stream = torch.cuda.current_stream()
    for graph in (True, False):
        spec = hd.make_run_spec(flags, "tanh", 0.0, use_graph=graph)
        for _ in range(5):
            hd.hd_run(st.h, spec, x1, out)
        torch.cuda.synchronize()
        reps = 200
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            hd.hd_run(st.h, spec, x1, out)
        e1.record(stream)
        torch.cuda.synchronize()
        res["us_per_product_graph" if graph else "us_per_product_stream"] = e0.elapsed_time(e1) * 1e3 / reps / T
    st.close()
    res.update({"config": "Gin(1000, 1000), entries N(0, 1/n), T=10, all Q, x_{t+1} = tanh(y_t), FP64",
                "value": float(n) * T * T / (res["us_per_product_graph"] * T * 1e-6), "unit": UNIT,
                "timing": "CUDA events around 200 back-to-back trajectories (hd_run), per product"})
    return res


def complex_phase(y):
    """Entrywise phase y / |y| (0 where y is 0): the dynamics of the complex workload."""
    import torch
    a = torch.abs(y)
    return torch.where(a > 0, y / torch.where(a > 0, a, torch.ones_like(a)), torch.zeros_like(y))


def measure_complex(args, rank, world, dist):
    """Complex ensemble (the paper's section "Other Random Matrix Ensembles"): Q ~ Haar on the
    unitary group U(n), n = 10^6, T = 100 products of Q, x_{t+1} = y_t / |y_t| entrywise,
    complex FP64 (hd_complex_apply, host-driven, the phase map in torch).  CUDA events around
    whole trajectories.  Algorithmic work: five passes of complex multiply-adds over the stacks
    per step (4 real FMAs each), 40 n k flops at k = t - 1.  All products are Q: under Q / Q^H
    alternation the phase map converges (the oracle's alpha_t / ||x_t|| falls to 1.5e-4 by
    step 20 at n = 2e4), after which every new reflector is built from rounding."""
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    n, T = 10 ** 6, 100
    st = hd.HDComplex("haar", n, n, T, args.seed, "f64", trial=rank)
    x1 = torch.complex(torch.tensor(synth.x1(n, args.seed, trial=rank)),
                       torch.tensor(synth.x1(n, args.seed + 7, trial=rank))).to("cuda")

    def run():
        st.reset()
        x = x1
        for t in range(1, T + 1):
            x = complex_phase(st.apply(x, False))
        return x

    run()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    secs = max_over_ranks(e0.elapsed_time(e1) / 1e3 / reps, dist)
    st.close()
    flops = 40.0 * n * T * (T - 1) / 2.0
    return {"value": job_throughput(float(n) * T * T, world, secs), "unit": UNIT, "ms_per_trajectory": secs * 1e3,
            "n": n, "T": T, "dtype": "c128 (complex FP64)",
            "fp64_TFLOPs": flops / secs / 1e12,
            "config": "Haar U(n), n=1e6, T=100, all Q, x_{t+1} = y_t / |y_t| entrywise",
            "timing": "CUDA events around 3 host-driven trajectories (hd_complex_apply, torch phase map)"}


FIG1A_N, FIG1A_K, FIG1A_TRIALS, FIG1A_CHUNK = 1000, 50, 100_000, 25_000


def measure_fig1a(args, rank, world, dist):
    """The paper's Fig. 1a experiment (Section 2.1) at its size: ISTA for the lasso on
    Gin(m, n), n = 1000, m = 500, entries N(0, 1/m), beta* ~ 0.2 delta_0 + 0.8 N(0, 2^2),
    w ~ N(0, 0.1^2), tau = 0.3, threshold 0.6, 50 iterations, over 10^5 independent trials:
    the mean MSE (1/n) ||x^k - beta*||^2 per iteration with its standard error.  Batched HD
    ISTA (hd_run with HD_DYN_ISTA, FP32 storage, one graph per chunk of 25,000 trials); x^k
    recorded per step (x_record) and reduced on the GPU.  Wall clock around all chunks,
    synchronised, including the per-chunk state creation and input uploads."""
    import numpy as np
    import torch
    import synth
    import paper_2101_07464_gb300 as hd
    n, K = FIG1A_N, FIG1A_K
    m, T = n // 2, 2 * FIG1A_K
    flags = [alt(t) for t in range(1, T + 1)]
    total = FIG1A_TRIALS
    s1 = np.zeros(K)
    s2 = np.zeros(K)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    run_secs = 0.0
    for c0 in range(0, total, FIG1A_CHUNK):
        cnt = min(FIG1A_CHUNK, total - c0)
        base = rank * total + c0
        b = hd.HDBatch("ginibre", [m] * cnt, [n] * cnt, T, args.seed, "f32", trial=base)
        b.set_trial_sigmas([m ** -0.5] * cnt)
        rng_b = synth.rng(args.seed, 10, base)
        beta = ((rng_b.random((cnt, n)) < 0.8) * 2.0 * rng_b.standard_normal((cnt, n))).astype(np.float32)
        w = (0.1 * synth.rng(args.seed, 11, base).standard_normal((cnt, m))).astype(np.float32)
        bt = torch.from_numpy(beta.reshape(-1)).cuda()
        wt = torch.from_numpy(w.reshape(-1)).cuda()
        xrec = torch.zeros((T, n * cnt), dtype=torch.float32, device="cuda")
        out = torch.empty(n * cnt, dtype=torch.float32, device="cuda")
        spec = hd.make_run_spec(flags, "ista", 0.6, use_graph=True, aux=wt, x_record=xrec, b=0.3)
        torch.cuda.synchronize()
        r0 = time.perf_counter()
        hd.hd_run(b.h, spec, bt, out)
        torch.cuda.synchronize()
        run_secs += time.perf_counter() - r0
        xs = xrec[1::2].reshape(K, cnt, n).double()
        mse = ((xs - bt.double().reshape(1, cnt, n)) ** 2).mean(dim=2)
        s1 += mse.sum(dim=1).cpu().numpy()
        s2 += (mse ** 2).sum(dim=1).cpu().numpy()
        del xrec, xs, mse
        b.close()
    secs = max_over_ranks(time.perf_counter() - t0, dist)
    mean = s1 / total
    se = np.sqrt(np.maximum(s2 / total - mean ** 2, 0.0) / (total - 1))
    return {"trials": total * world, "n": n, "m": m, "iterations": K, "products": T, "dtype": "f32",
            "seconds": secs, "seconds_in_hd_run": run_secs,
            "mse_per_iteration": [_g3(v) for v in mean], "se_per_iteration": [_g3(v) for v in se],
            "value": job_throughput(float(total) * n * T * T, world, run_secs), "unit": "trials*n*T^2/s",
            "config": "Fig. 1a: lasso ISTA on Gin(n/2, n), n=1000, entries N(0, 1/m), 50 iterations, tau=0.3, "
                      "threshold 0.6, beta* ~ 0.2 delta_0 + 0.8 N(0, 4), w ~ N(0, 0.01), 10^5 trials "
                      "(chunks of 25,000 in one batched state each)",
            "timing": "wall clock, synchronised: seconds covers state creation, inputs and reductions; "
                      "seconds_in_hd_run the hd_run calls alone (value uses the latter)"}


def roofline_of(prof, dtype, n, T, peaks):
    """Roofline of the dominant sweep (largest total time inside the timed trajectories):
    FP64 against the measured FP64 FMA rate (algorithmic flops), FP32 against the measured
    HBM copy rate (algorithmic bytes).  Times are CUDA events on the launching stream."""
    dom = max(prof, key=lambda k: prof[k][0])
    ms, nl, by = prof[dom]
    per_kernel = {k: {"ms_total": v[0], "launches": v[1], "GBps": (v[2] / (v[0] / 1e3) / 1e9) if v[0] else None}
                  for k, v in prof.items()}
    # every step of a trajectory launches either the step kernel or an update sweep
    trajectories = (prof["update"][1] + prof.get("step", (0, 0, 0))[1]) / T
    cols = haar_columns(T, round(prof.get("step", (0, 0, 0))[1] / trajectories) if trajectories else 0)
    if dtype == "f64":
        flops = FLOPS_PER_ELEMENT[dom] * n * cols[dom] * trajectories
        achieved = (flops / nl) / ((ms / nl) / 1e3) / 1e12 if nl else 0.0
        for k, v in prof.items():
            if v[0] and v[1]:
                per_kernel[k]["TFLOPs"] = FLOPS_PER_ELEMENT[k] * n * cols[k] * trajectories / (v[0] / 1e3) / 1e12
        r = {"bound": "alu", "kernel": KERNEL_NAME[dom], "achieved": achieved, "peak": peaks["fp64_tflops"],
             "unit": "TFLOP/s", "frac": achieved / peaks["fp64_tflops"],
             "peak_source": "measured now on this GPU: hd_fp64_fma_rate (8 independent FMA chains per "
                            "thread, 8 CTAs of 256 threads per SM, best of 5 event-timed launches)",
             "work": "%g FP64 flops per stack element (2 per FMA) x n x the columns of each launch "
                     "(t - 1 before step t)" % FLOPS_PER_ELEMENT[dom],
             "traffic": ((by / nl) * TRAFFIC_RATIO["f64"] if (nl and dom == TRAFFIC_KERNEL and TRAFFIC_RATIO["f64"])
                         else None),
             "hbm_GBps": (by / nl) / ((ms / nl) / 1e3) / 1e9 if nl else None}
    else:
        achieved = (by / nl) / ((ms / nl) / 1e3) / 1e9 if nl else 0.0
        r = {"bound": "hbm", "kernel": KERNEL_NAME[dom], "achieved": achieved, "peak": peaks["hbm_gbs"],
             "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["hbm_source"],
             "traffic": ((by / nl) * TRAFFIC_RATIO["f32"] if (nl and dom == TRAFFIC_KERNEL and TRAFFIC_RATIO["f32"])
                         else None)}
    if r["traffic"] is not None:
        r["traffic_source"] = TRAFFIC_SOURCE
    r["timing"] = ("CUDA events on the launching stream around every sweep, recorded in a second pass "
                   "of the same trajectories (events inside the graph would perturb the headline timing)")
    r["per_kernel"] = per_kernel
    return r


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
    hbm, hbm_kind = measured_peaks()
    peaks = {"hbm_gbs": hbm, "hbm_source": hbm_kind, "fp64_tflops": fp64_peak()}

    def measure(dtype, profile):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        st = hd.HD("haar", n, n, T, args.seed, dtype, trial=rank)
        if args.step_kernel:
            hd.hd_set_engine(st.h, step_kernel=True)
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
    roofline = roofline_of(prof, args.dtype, n, T, peaks)
    credited = 2.0 * n * tdt.itemsize * T * (T + 1) / 2.0 * world

    side = None
    other = "f32" if args.dtype == "f64" else "f64"
    if not args.no_side:
        st2, _, secs2, prof2, _ = measure(other, profile=True)
        st2.close()
        ps = secs2 / args.steps
        side = {"value": units / ps, "unit": UNIT, "ms_per_step": ps * 1e3, "dtype": other,
                "storage": "FP32 stacks and vectors, FP64 coefficients and cross-thread sums" if other == "f32"
                else "FP64",
                "step_credited_GBps": 2.0 * n * (4 if other == "f32" else 8) * T * (T + 1) / 2.0 * world / ps / 1e9,
                "roofline": roofline_of(prof2, other, n, T, peaks)}

    c1 = None
    if not args.no_c1:
        c1 = measure_c1(args)
    stepk = None
    if not args.no_side:
        stepk = measure_step_kernel(args, rank)
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
    cplx = None
    if not args.no_complex:
        try:
            cplx = measure_complex(args, rank, world, dist)
        except Exception as exc:   # reported in the line, the headline stands
            cplx = {"error": "%s: %s" % (type(exc).__name__, exc)}
    fig1a = None
    if not args.no_fig1a:
        try:
            fig1a = measure_fig1a(args, rank, world, dist)
        except Exception as exc:   # reported in the line, the headline stands
            fig1a = {"error": "%s: %s" % (type(exc).__name__, exc)}
    large = None
    if not args.no_large:
        try:
            large = measure_large(args, rank, world, dist)
        except Exception as exc:   # reported in the line, the headline stands
            large = {"error": "%s: %s" % (type(exc).__name__, exc)}

    # the CPU-baseline leg (N = 1 only: the oracle is a single-host baseline), then the
    # accuracy of every result against the oracle's reference values
    cpu, accuracy = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, refs = cpu_baseline_leg(args, n, T, not args.no_accuracy)
        if not args.no_accuracy:
            hr = refs["headline"]
            acc64 = accuracy_haar_sign("f64", n, T, args.seed, (hr["xs"], hr["ys"], hr["fs"]),
                                       (hr["xs"], hr["ys"], hr["fs"]))
            fx = refs["fp32"]
            acc32 = accuracy_haar_sign("f32", fx["n"], T, args.seed, fx["teacher"], fx["free"])
            acc32["note"] = ("reduced n; teacher-forced inputs are the oracle's rounded to FP32, the "
                             "free run is against the oracle's FP64 trajectory")
            accuracy = acc64 if args.dtype == "f64" else acc32
            if side is not None:
                side["accuracy"] = acc32 if other == "f32" else acc64
            if c1 is not None:
                c1["accuracy"] = accuracy_c1(refs["c1"], args.seed)
            if amp is not None:
                amp["accuracy"] = accuracy_amp(refs["amp"], args.seed)
            if adj is not None:
                adj["accuracy"] = accuracy_grad("adjoint", refs["adjoint"], args.seed)
            if ista is not None and "error" not in ista:
                ista["accuracy"] = accuracy_grad("ista", refs["ista"], args.seed)
            if paper_ista is not None and "seconds" in paper_ista:
                paper_ista["accuracy"] = {"n": refs["paper_ista"]["n"], "products": accuracy_products(refs["paper_ista"], "f64"),
                                          "how": "reduced n, FP64, every product teacher-forced (hd_apply on the oracle's inputs)"}
            if spectral is not None and "seconds" in spectral:
                spectral["accuracy"] = {"n": refs["spectral"]["n"] // 2,
                                        "products": accuracy_products(refs["spectral"], "f64"),
                                        "how": "reduced n, FP64, 30 power iterations, every product teacher-forced"}
            if large is not None and "forward" in large:
                large["accuracy"] = accuracy_large(refs["large"], args.seed)
            if cplx is not None and "value" in cplx:
                cplx["accuracy"] = accuracy_complex(refs["complex"])
            if fig1a is not None and "mse_per_iteration" in fig1a:
                import numpy as np
                d = refs["fig1a"]
                hm = np.array(fig1a["mse_per_iteration"])
                hs = np.array(fig1a["se_per_iteration"])
                z = np.abs(hm - d["mean"]) / np.sqrt(hs ** 2 + d["se"] ** 2)
                fig1a["accuracy"] = {"direct_trials": d["trials"], "direct_mse_per_iteration": [_g3(v) for v in d["mean"]],
                                     "max_gap_in_combined_se": _g3(z.max()),
                                     "how": "HD's mean MSE per iteration against the direct approach (dense "
                                            "Gin(n/2, n) per trial, oracle/direct.py, same n) over its trials; "
                                            "gap in units of the combined standard error"}
        del refs

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
                           "engine": ("step kernel (one launch per step)" if args.step_kernel
                                      else "two launches per step (update sweep, fused output sweep)"),
                           "launch_shapes": "built-in" if args.no_autotune
                           else "hd_autotune (untimed, before the timed region)"},
                "roofline": roofline,
                "step_credited_GBps": credited / per_step / 1e9,
                "accuracy": accuracy,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, other: side, "c1": c1, "step_kernel": stepk, "batched_amp": amp, "adjoint": adj, "ista": ista,
                "paper_ista": paper_ista, "spectral": spectral, "complex": cplx, "fig1a": fig1a, "large": large}
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
