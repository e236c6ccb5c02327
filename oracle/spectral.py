"""The spectral method of the paper's Section 2.2 on Householder Dice (test infrastructure).

Sensing matrix A = [I_n 0] Q (eq. A_ortho) with Q ~ Haar(m), m = floor(alpha n), alpha > 1:
its columns are the sensing vectors a_i in R^n.  Measurements y_i = tanh(|a_i^T xi|), i.e.
y = tanh(|Q^T [xi; 0]|), and D = (1/m) A diag(y) A^T (eq. D_mtx), so

    D x = (1/m) [I_n 0] Q (y o (Q^T [x; 0])):

one Q^T and one Q product of the Householder Dice state per multiplication by D.  The
leading eigenvector is found by power iteration, x_{k+1} = D x_k / ||D x_k|| (the paper uses
Krylov-Schur; both only multiply by D).  Products: Q^T [xi; 0], then Q^T, Q per iteration.
"""
import torch

F64 = torch.float64


def pad(x, m):
    x = torch.as_tensor(x, dtype=F64)
    return torch.cat([x, torch.zeros(m - x.shape[0], dtype=F64)])


def measurements(ora, xi, m):
    """y = tanh(|A^T xi|) from one Q^T product of the oracle `ora` (Haar(m))."""
    return torch.tanh(torch.abs(ora.apply(pad(xi, m), True)))


def apply_D(ora, y, x, n, m):
    """D x = (1/m) [I 0] Q (y o Q^T [x; 0]) (two products)."""
    u = ora.apply(pad(x, m), True)
    return ora.apply(y * u, False)[:n] / m


def power_iteration(ora, xi, n, m, K, x0):
    """Measurements, then K normalised power iterations from x0; returns (y, [x_1 .. x_K])."""
    y = measurements(ora, xi, m)
    x = torch.as_tensor(x0, dtype=F64)
    x = x / torch.linalg.vector_norm(x)
    xs = []
    for _ in range(K):
        v = apply_D(ora, y, x, n, m)
        x = v / torch.linalg.vector_norm(v)
        xs.append(x)
    return y, xs
