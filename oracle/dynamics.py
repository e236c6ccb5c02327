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


def run_trace(state, x1, T, f, schedule, cast=None):
    """Iterate eq. (dynamics) for T steps, x_0 = 0, recording what each product consumed.

    cast (optional) rounds x_1 and every result of f before the next product uses it, so that
    a lower-precision implementation can be handed exactly the same inputs (teacher forcing).
    Returns (xs, ys, fs): xs[t-1] = x_t as fed to product t, ys[t-1] = M_t x_t and
    fs[t-1] = f's result after step t, before rounding.  x_{t-1} enters f as the zero vector
    of y_t's space when its own dimension differs (first step of a rectangular schedule).
    """
    c = cast if cast is not None else (lambda v: np.asarray(v, dtype=np.float64))
    x = c(x1)
    x_prev = np.zeros_like(x)
    xs, ys, fs = [], [], []
    for t in range(1, T + 1):
        y = np.asarray(state.apply(x, transpose=schedule(t)), dtype=np.float64)
        xp = x_prev if x_prev.shape == y.shape else np.zeros_like(y)
        fx = f(y, x, xp)
        xs.append(x)
        ys.append(y)
        fs.append(fx)
        x_prev, x = x, c(fx)
    return xs, ys, fs


def soft_threshold(r, theta):
    return np.sign(r) * np.maximum(np.abs(r) - theta, 0.0)


def amp_trace(state, beta, w, T, thr=1.1, cast=None):
    """T products of AMP for the linear model y = Q beta + w, Q in R^{m x n}, step by step.

    Product 1 is Q beta (then y = Q beta + w, z^0 = y, x^0 = 0); after that the products
    alternate Q^T z^k (even t) and Q x^{k+1} (odd t):
        x^{k+1} = eta(x^k + Q^T z^k; theta_k),  theta_k = thr * ||z^k|| / sqrt(m)
        z^{k+1} = y - Q x^{k+1} + z^k ||x^{k+1}||_0 / m      (the Onsager term)
    with eta the soft threshold.  cast (optional) rounds each updated vector before anything
    uses it (teacher forcing of a lower-precision implementation); y keeps full precision.
    Returns a dict of per-step lists: products[t-1] = the t-th product, updates[t-1] = the
    vector step t updates (z^0, x^1, z^1, x^2, ...) and used[t-1] = that vector after cast.
    """
    c = cast if cast is not None else (lambda v: v)
    beta = np.asarray(beta, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    m = w.shape[0]
    q = np.asarray(state.apply(beta, transpose=False), dtype=np.float64)
    y = q + w
    z = c(y.copy())
    x = np.zeros_like(beta)
    tr = {"products": [q], "updates": [y.copy()], "used": [z]}
    for t in range(2, T + 1):
        if t % 2 == 0:
            s = np.asarray(state.apply(z, transpose=True), dtype=np.float64)
            x_new = soft_threshold(x + s, thr * np.linalg.norm(z) / np.sqrt(m))
            tr["products"].append(s)
            tr["updates"].append(x_new)
            x = c(x_new)
            tr["used"].append(x)
        else:
            q = np.asarray(state.apply(x, transpose=False), dtype=np.float64)
            z_new = y - q + z * (np.count_nonzero(x) / m)
            tr["products"].append(q)
            tr["updates"].append(z_new)
            z = c(z_new)
            tr["used"].append(z)
    return tr


def ista_trace(state, beta, w, T, theta, tau, cast=None):
    """T products of ISTA for the lasso (Section 2.1): y = Q beta + w, x^0 = 0, and
        x^{k+1} = eta(x^k + tau Q^T (y - Q x^k); theta),
    as products: Q beta (t = 1), then Q^T z^k (even t, z^k = y - Q x^k; z^0 = y because
    x^0 = 0, so Q x^0 is not formed) and Q x^{k+1} (odd t).  theta is the threshold
    (lambda tau in the paper's notation).  cast and the returned lists are as in amp_trace:
    products, updates (z^0, x^1, z^1, x^2, ...) and the updates after cast."""
    c = cast if cast is not None else (lambda v: v)
    beta = np.asarray(beta, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    q = np.asarray(state.apply(beta, transpose=False), dtype=np.float64)
    y = q + w
    z = c(y.copy())
    x = np.zeros_like(beta)
    tr = {"products": [q], "updates": [y.copy()], "used": [z]}
    for t in range(2, T + 1):
        if t % 2 == 0:
            s = np.asarray(state.apply(z, transpose=True), dtype=np.float64)
            x_new = soft_threshold(x + tau * s, theta)
            tr["products"].append(s)
            tr["updates"].append(x_new)
            x = c(x_new)
            tr["used"].append(x)
        else:
            q = np.asarray(state.apply(x, transpose=False), dtype=np.float64)
            z_new = y - q
            tr["products"].append(q)
            tr["updates"].append(z_new)
            z = c(z_new)
            tr["used"].append(z)
    return tr


def amp(state, beta, w, T, thr=1.1):
    """T products of AMP (amp_trace without rounding).  Returns (xs, zs): the x^k after each
    Q^T product and the z^k (z^0 first)."""
    tr = amp_trace(state, beta, w, T, thr)
    xs = [v for t, v in enumerate(tr["used"], start=1) if t % 2 == 0]
    zs = [v for t, v in enumerate(tr["used"], start=1) if t % 2 == 1]
    return xs, zs
