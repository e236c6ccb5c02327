"""Helpers shared by the GPU parity tests: teacher-forced comparison of the CUDA path with
the oracle (both get the same x_t; the error of each step is ||y_gpu - y_oracle|| / ||y_oracle||)."""
import numpy as np

import synth
from oracle.hd import make_oracle

TOL = {"f64": 1e-12, "f32": 1e-5}


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
