"""Other ensembles built from the Gaussian and Haar oracles (test infrastructure only).

Paper, section "Other Random Matrix Ensembles":
  * GOE(n): W = (Q + Q^T)/sqrt(2) with Q ~ Gin(n, n) is GOE(n); a product W x is simulated by
    the two products y_hat = Q x and Q^T x of one Householder Dice state, y = (Q^T x + y_hat)/sqrt(2).
  * eq. (inv): Q = U Sigma V with U ~ Haar(m), V ~ Haar(n) independent and Sigma an m x n
    rectangular diagonal matrix; Householder Dice runs one state per orthogonal factor.
"""
import math

import torch

from .hd import GinibreOracle, HaarOracle

F64 = torch.float64


def goe_apply(gin, x):
    """W x for the square Ginibre oracle `gin` (two of its products, Q x first)."""
    yhat = gin.apply(x, False)
    return (gin.apply(x, True) + yhat) / math.sqrt(2.0)


def sigma_apply(s, v, m_out):
    """The rectangular diagonal Sigma (diagonal s) times v, into R^{m_out}."""
    v = torch.as_tensor(v, dtype=F64)
    k = min(len(s), v.shape[0], m_out)
    out = torch.zeros(m_out, dtype=F64)
    out[:k] = torch.tensor([float(a) for a in s[:k]], dtype=F64) * v[:k]
    return out


def usv_apply(U, V, s, x, transpose=False):
    """Q x for Q = U Sigma V (eq. inv), or Q^T x = V^T Sigma^T U^T x when transpose.
    U: HaarOracle on R^m, V: HaarOracle on R^n, s: the min(m, n) diagonal entries."""
    m, n = U.n, V.n
    if not transpose:
        return U.apply(sigma_apply(s, V.apply(x, False), m), False)
    return V.apply(sigma_apply(s, U.apply(x, True), n), True)


def make_goe(n, T, seed, trial=0, sigma=1.0):
    return GinibreOracle(n, n, T, seed, trial=trial, sigma=sigma)


def make_usv(m, n, T, seed_u, seed_v):
    return HaarOracle(m, T, seed_u), HaarOracle(n, T, seed_v)
