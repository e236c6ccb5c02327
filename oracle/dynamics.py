"""Caller-side dynamics f_t of eq. (dynamics) for the synthetic workloads (test infrastructure).

The paper leaves f_t to the caller (eq. dynamics, Section 1).  These are the oracle's own
plain numpy versions of the workloads' update rules; the CUDA path has its own kernels for
them and shares nothing with this file.

  tanh       x_{t+1} = tanh(y_t)                                (Ginibre, all Q)
  sign_mem   x_{t+1} = sign(y_t) + 0.5 x_{t-1}, x_0 = 0, sign(0) = 0   (Haar, Q / Q^T alternating)
  norm_tanh  x_{t+1} = normalize(tanh(y_t) + 0.1 x_t)          (Haar, all Q)
  amp        approximate message passing for y = Q beta + w (the AMP family the paper
             lists among its target dynamics in Section 1), soft threshold 1.1 sigma_t
The schedule helpers return the transpose flag of step t (1-based).
"""
import numpy as np


def schedule_all_q(t):
    return False


def schedule_alternating(t):
    """Q at odd t, Q^T at even t."""
    return t % 2 == 0


def f_tanh(y, x_t, x_prev):
    return np.tanh(y)


def f_sign_mem(y, x_t, x_prev):
    return np.sign(y) + 0.5 * x_prev


def f_norm_tanh(y, x_t, x_prev):
    v = np.tanh(y) + 0.1 * x_t
    return v / np.sqrt(np.dot(v, v))


DYNAMICS = {"tanh": f_tanh, "sign_mem": f_sign_mem, "norm_tanh": f_norm_tanh}
SCHEDULES = {"all_q": schedule_all_q, "alternating": schedule_alternating}


def run(state, x1, T, f, schedule, x0=None):
    """Iterate eq. (dynamics) for T steps on any state with apply(x, transpose).

    Returns (xs, ys): xs[0] = x_1 ... xs[T] = x_{T+1}; ys[t-1] = M_t x_t.
    """
    x_prev = np.zeros_like(np.asarray(x1, dtype=np.float64)) if x0 is None else np.asarray(x0)
    x = np.asarray(x1, dtype=np.float64)
    xs, ys = [x], []
    for t in range(1, T + 1):
        y = np.asarray(state.apply(x, transpose=schedule(t)), dtype=np.float64)
        x_next = f(y, x, x_prev)
        ys.append(y)
        x_prev, x = x, x_next
        xs.append(x)
    return xs, ys


def soft_threshold(r, theta):
    return np.sign(r) * np.maximum(np.abs(r) - theta, 0.0)


def amp(state, beta, w, T, thr=1.1):
    """T products of AMP for the linear model y = Q beta + w, Q in R^{m x n}.

    Product 1 is Q beta (then y = Q beta + w, z^0 = y, x^0 = 0); after that the products
    alternate Q^T z^k (even t) and Q x^{k+1} (odd t):
        x^{k+1} = eta(x^k + Q^T z^k; theta_k),  theta_k = thr * ||z^k|| / sqrt(m)
        z^{k+1} = y - Q x^{k+1} + z^k ||x^{k+1}||_0 / m      (the Onsager term)
    with eta the soft threshold.  Returns (xs, zs): the x^k after each Q^T product and the
    z^k (z^0 first).
    """
    beta = np.asarray(beta, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    m = w.shape[0]
    y = np.asarray(state.apply(beta, transpose=False), dtype=np.float64) + w
    z = y.copy()
    x = np.zeros_like(beta)
    xs, zs = [], [z]
    for t in range(2, T + 1):
        if t % 2 == 0:
            r = x + np.asarray(state.apply(z, transpose=True), dtype=np.float64)
            x = soft_threshold(r, thr * np.linalg.norm(z) / np.sqrt(m))
            xs.append(x)
        else:
            q = np.asarray(state.apply(x, transpose=False), dtype=np.float64)
            z = y - q + z * (np.count_nonzero(x) / m)
            zs.append(z)
    return xs, zs
