"""Pathwise derivatives of oracle trajectories (test infrastructure only).

The oracle applies every reflector with torch float64 CPU ops, takes the sign of each
reflector from a detached value, and treats the Gaussian draws as constants.  So torch
autograd of a trajectory computed with it is the derivative of the sampler's output with the
draws held fixed, the quantity the library's reverse mode computes.  The paper has no
gradients: this is the plain chain rule through Algorithms 1 and 2 as the oracle states them.
"""
import torch

from .hd import make_oracle


def trajectory(ensemble, m, n, T, seed, schedule, f, x1, params=(), trial=0, sigma=1.0):
    """x_{T+1} of x_{t+1} = f(t, y_t, x_t, x_{t-1}, *params), y_t = M_t x_t (M_t = Q^T where
    schedule[t-1] is true), on the oracle of (ensemble, m, n, T, seed, trial, sigma).
    x_{t-1} is None at t = 1.  Differentiable in x1 and params by torch autograd."""
    ora = make_oracle(ensemble, m, n, T, seed, trial=trial, sigma=sigma)
    x, xprev = x1, None
    for t in range(1, T + 1):
        y = ora.apply(x, bool(schedule[t - 1]))
        x, xprev = f(t, y, x, xprev, *params), x
    return x
