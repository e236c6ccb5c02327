"""Helpers shared by the GPU parity tests: teacher-forced comparison of the CUDA path with
the oracle (both get the same x_t; the error of each step is ||y_gpu - y_oracle|| / ||y_oracle||)."""
import numpy as np

import synth
from oracle.hd import make_oracle

TOL = {"f64": 1e-12, "f32": 1e-5}
# Smallest alpha_t / ||x_t|| (the part of a step's input that the revealed reflectors do not
# already fix) at which per-step parity is meaningful: the unit roundoff over the tolerance.
# Below it the new reflector is built from a tail dominated by rounding (reading A13(i)).
COND_MIN = {"f64": 1.1e-16 / 1e-12, "f32": 6.0e-8 / 1e-5}


def next_input(y, t_next, transpose_next, m, n, seed):
    """tanh of the output when its dimension fits the next product, else a fresh seeded vector."""
    want = m if transpose_next else n
    if y.shape[0] == want:
        return np.tanh(y)
    return synth.x1(want, seed, trial=1000 + t_next)


def teacher_forced(ens, m, n, T, seed, dtype, schedule, sigma=1.0, x1=None, dynamics=None,
                   trial=0, setup=None):
    """setup(state): called on the GPU state once, before its first product."""
    import torch
    from paper_2101_07464_gb300 import HD
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ora = make_oracle(ens, m, n, T, seed, trial=trial, sigma=sigma)
    gpu = HD(ens, m, n, T, seed, dtype, sigma=sigma, trial=trial)
    if setup is not None:
        setup(gpu)
    x = synth.x1(m if schedule(1) else n, seed) if x1 is None else x1
    x_prev = None
    errs = []
    try:
        for t in range(1, T + 1):
            tr = schedule(t)
            x = np.asarray(x, dtype=np.float64)
            if dtype == "f32":
                x = x.astype(np.float32).astype(np.float64)
            yo = ora.apply(x, tr).numpy()
            yg = gpu.apply(torch.tensor(x, dtype=tdt, device="cuda"), tr).double().cpu().numpy()
            den = np.linalg.norm(yo)
            errs.append(np.linalg.norm(yg - yo) / den if den > 0 else np.linalg.norm(yg))
            if dynamics is not None:
                xn = dynamics(yo, x, x_prev)
            else:
                xn = next_input(yo, t + 1, schedule(t + 1), m, n, seed)
            x_prev, x = x, xn
    finally:
        gpu.close()
    return np.array(errs)


def f32_cast(v):
    """Round a float64 vector to the nearest FP32 values (kept as float64)."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def oracle_trajectory(ens, m, n, T, seed, schedule, f, x1, sigma=1.0, cast=None, trial=0):
    """The oracle's own trajectory (oracle.dynamics.run_trace on a fresh oracle state):
    (xs, ys, fs) with xs[t-1] = x_t as fed to product t, ys[t-1] = y_t and fs[t-1] = f's
    result after step t before rounding by cast."""
    from oracle.dynamics import run_trace
    ora = make_oracle(ens, m, n, T, seed, trial=trial, sigma=sigma)
    return run_trace(ora, x1, T, f, schedule, cast=cast)


def elem_err(a, b, head):
    """Element-wise error of one step's output: rows below `head` (the pivot rows that the
    step's reflectors have fixed, t of them after step t) relative to ||b||_2, the other rows
    relative to max_i |b_i|.  The oracle forms each pivot row by applying eq. Householder
    literally, as the difference of two terms of the size of ||x_t|| (H(a) a = ||a|| e_1), so
    its own rounding there scales with the vector norm and the length of its dot products
    (1.2e-11 absolute at n = 10^6, ||x|| = 10^3, with the GPU host's BLAS); the other rows
    carry rounding on the scale of the entries."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a - b)
    h = min(int(head), b.shape[0])
    tail = d[h:].max() / np.abs(b).max() if h < b.shape[0] else 0.0
    hd_ = d[:h].max() / np.linalg.norm(b) if h > 0 else 0.0
    return float(max(tail, hd_))


def max_rel(a, b):
    """max_i |a_i - b_i| / max_i |b_i| (element-wise error on the scale of the vector)."""
    b = np.asarray(b, dtype=np.float64)
    s = np.abs(b).max()
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / s) if s > 0 else float(np.abs(a).max())
