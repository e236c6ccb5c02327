"""Dynamics shared by the ISTA tests: ISTA (Section 2.1 of the paper, A = Q square Gaussian)
as products of Householder Dice, in the trajectory API's f_t form."""
import torch


def ista_schedule(K):
    """t = 1: Q beta*; then Q x^k and Q^T r^k alternate (2K + 1 products)."""
    return [False] + [bool(t % 2) for t in range(2, 2 * K + 2)]


def ista_f(w):
    """f_t(y_t, x_t, x_{t-1}; theta, tau) for y = Q beta* + w, x^0 = 0,
    x^{k+1} = eta(x^k + tau Q^T (y - Q x^k); theta_k), eta the soft threshold.
    Keeps y from the first product."""
    store = {}

    def f(t, y, x, xprev, theta, tau):
        if t == 1:
            store["y"] = (y + w).detach()
            return torch.zeros_like(y)
        if t % 2 == 0:                      # y = Q x^k: next input r^k = y_obs - Q x^k
            return store["y"] - y
        k = (t - 3) // 2                    # y = Q^T r^k, xprev = x^k
        v = xprev + tau * y
        return torch.sign(v) * torch.clamp(v.abs() - theta[k], min=0.0)
    return f
