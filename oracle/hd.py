"""Plain CPU FP64 oracle of Householder Dice (test infrastructure only).

This is a slow, literal restatement of the paper's method, used by the tests, by
`__graft_entry__.smoke()` and by the CPU-baseline leg of `bench.py` to check and time the
CUDA path.  The product path never imports it.

What it follows:
  * the reflector H(v) of eq. (Householder) with the reading sign(v1) = +1 for v1 >= 0 and
    -1 otherwise (the printed "0 otherwise" would make H singular, contradicting
    H in O(n) stated right after it, and the complex reflector of eq. (Householder_c)
    reduces to this choice for real v);
  * the generalised reflector H_k(p) of eq. (Householder_e), identity when p[k:n] = 0;
  * Algorithm 1 (Ginibre, Section 3.2) and Algorithm 2 (Haar, Section 3.3), step by
    step in the paper's order.  Products of reflectors are applied one reflector at a
    time by the defining formula; there is no blocked (WY) form here.
Indices are 0-based in code: the paper's H_k acts on code indices k-1 .. n-1.

Everything is torch float64 on the CPU so that torch autograd can differentiate a
trajectory (the random draws are constants).  The Gaussian draws come from the oracle's
own Philox copy in `oracle.philox`.
"""
import numpy as np
import torch

from . import philox

F64 = torch.float64


def _vec(x):
    if isinstance(x, torch.Tensor):
        return x.to(F64)
    return torch.as_tensor(np.asarray(x, dtype=np.float64))


class Reflector:
    """The generalised Householder reflector H_{k+1}(p) (0-based pivot k), eq. (Householder_e).

    H(a) = -s (I - 2 u u^T / u^T u) with u = a + s ||a|| e_1, s = sign(a_1), eq. (Householder);
    it is symmetric and orthogonal, H(a) e_1 = a/||a|| and H(a) a = ||a|| e_1
    (eq. Householder_property).  On the first k coordinates it is the identity.
    """

    def __init__(self, k, p):
        p = _vec(p)
        a = p[k:]
        self.k = k
        self.alpha = torch.sqrt(torch.dot(a, a))
        self.identity = bool(self.alpha.detach() == 0)
        if self.identity:
            self.s = 1.0
            self.u = None
            self.uu = None
            return
        self.s = 1.0 if float(a[0].detach()) >= 0.0 else -1.0
        e1 = torch.zeros_like(a)
        e1[0] = 1.0
        self.u = a + self.s * self.alpha * e1
        self.uu = torch.dot(self.u, self.u)

    def apply(self, w):
        """Return H_{k+1}(p) w for a vector w (w itself is not modified)."""
        w = _vec(w)
        if self.identity:
            return w.clone()
        head = w[:self.k]
        seg = w[self.k:]
        seg = -self.s * (seg - (2.0 * torch.dot(self.u, seg) / self.uu) * self.u)
        return torch.cat([head, seg])

    def dense(self, dim):
        """The dim x dim matrix (small cases only)."""
        eye = torch.eye(dim, dtype=F64)
        return torch.stack([self.apply(eye[:, j]) for j in range(dim)], dim=1)


def unit(dim, k):
    e = torch.zeros(dim, dtype=F64)
    e[k] = 1.0
    return e


def apply_in_order(refls, w):
    """refls[-1] ... refls[1] refls[0] w  (the first reflector acts first)."""
    for h in refls:
        w = h.apply(w)
    return w


def apply_reversed(refls, w):
    """refls[0] refls[1] ... refls[-1] w  (the last reflector acts first)."""
    for h in reversed(refls):
        w = h.apply(w)
    return w


class HaarOracle:
    """Algorithm 2: y_t = M_t x_t for Q ~ Haar(n), M_t in {Q, Q^T} chosen per step."""

    def __init__(self, n, T_max, seed, trial=0):
        if n <= 0:
            raise ValueError("n must be positive")
        if T_max > n:
            raise ValueError("Algorithm 2 requires T <= n")
        self.n, self.T_max, self.seed, self.trial = n, T_max, seed, trial
        self.reset(seed)

    def reset(self, seed=None):
        if seed is not None:
            self.seed = seed
        self.t = 0
        self.R = []   # R_1 .. R_t
        self.L = []   # L_1 .. L_t
        self.g = []   # the draws g_t (head entries 1..t-1 zero: never used by H_t(g_t))

    def draw(self, t):
        return torch.as_tensor(philox.gaussian_vector(self.seed, self.trial, t, self.n, t - 1))

    def apply(self, x, transpose=False):
        t = self.t + 1
        if t > self.T_max:
            raise ValueError("step would exceed T_max")
        x = _vec(x)
        g = self.draw(t)
        k = t - 1                      # pivot of H_t, 0-based
        if not transpose:
            p = apply_in_order(self.R, x)            # p_t = R_{t-1} ... R_1 x_t  (eq. pt)
            Rt, Lt = Reflector(k, p), Reflector(k, g)  # R_t = H_t(p_t), L_t = H_t(g_t)
            self.R.append(Rt)
            self.L.append(Lt)
            y = apply_reversed(self.L, Rt.apply(p))   # y_t = L_1 ... L_t R_t p_t
        else:
            p = apply_in_order(self.L, x)            # p_t = L_{t-1} ... L_1 x_t
            Lt, Rt = Reflector(k, p), Reflector(k, g)  # L_t = H_t(p_t), R_t = H_t(g_t)
            self.L.append(Lt)
            self.R.append(Rt)
            y = apply_reversed(self.R, Lt.apply(p))   # y_t = R_1 ... R_t L_t p_t
        self.g.append(g)
        self.t = t
        return y

    def probe(self, x, transpose=False):
        """Q^(t) x on the revealed part, without adding a step (eq. H_t).

        Returns (y, unrevealed) where unrevealed = ||entries t+1..n of R_t...R_1 x|| (or of
        L_t...L_1 x for Q^T): when it is zero, x never meets Q_{n-t} and y is exact.
        """
        x = _vec(x)
        t = self.t
        first, second = (self.R, self.L) if not transpose else (self.L, self.R)
        q = apply_in_order(first, x)
        unrevealed = torch.sqrt(torch.dot(q[t:], q[t:]))
        q = torch.cat([q[:t], torch.zeros(self.n - t, dtype=F64)])
        return apply_reversed(second, q), unrevealed

    def dense(self):
        """L_1..L_t R_t..R_1 as a dense matrix; equals Q exactly once t = n (small n only)."""
        eye = torch.eye(self.n, dtype=F64)
        cols = [apply_reversed(self.L, apply_in_order(self.R, eye[:, j])) for j in range(self.n)]
        return torch.stack(cols, dim=1)


class GinibreOracle:
    """Algorithm 1: y_t = M_t x_t for Q ~ Gin(m, n) with entries sigma * N(0, 1).

    sigma scales every new draw g_t; each term of y_t is linear in exactly one draw, so
    this is Q for the ensemble with entry variance sigma^2 (sigma = 1 is the paper's
    Gin(m, n)).
    """

    def __init__(self, m, n, T_max, seed, trial=0, sigma=1.0):
        if m <= 0 or n <= 0:
            raise ValueError("m and n must be positive")
        if T_max > min(m, n):
            raise ValueError("Algorithm 1 requires T <= min(m, n)")
        self.m, self.n, self.T_max = m, n, T_max
        self.seed, self.trial, self.sigma = seed, trial, sigma
        self.reset(seed)

    def reset(self, seed=None):
        if seed is not None:
            self.seed = seed
        self.t = self.r = self.l = 0
        self.R, self.L = [], []       # reflectors on R^n and on R^m
        self.u, self.v = [], []       # basis vectors u_i in R^m, v_i in R^n
        self.qstep = []               # True where step i used Q, False for Q^T

    def apply(self, x, transpose=False):
        t = self.t + 1
        if t > self.T_max:
            raise ValueError("step would exceed T_max")
        x = _vec(x)
        if not transpose:
            self.r += 1
            # g_t ~ Gin(m, 1); only Z_{1:l} g_t enters, so entries 1..l are never drawn
            g = torch.as_tensor(philox.gaussian_vector(self.seed, self.trial, t, self.m,
                                                       self.l, self.sigma))
            p = apply_in_order(self.R, x)                    # R_{r-1} ... R_1 x_t
            self.R.append(Reflector(self.r - 1, p))          # R_r = H_r(p)
            u = apply_reversed(self.L, g)                    # L_1 ... L_l Z_{1:l} g_t
            v = apply_reversed(self.R, unit(self.n, self.r - 1))  # R_1 ... R_r e_r
            self.u.append(u)
            self.v.append(v)
            y = torch.zeros(self.m, dtype=F64)
            for ui, vi in zip(self.u, self.v):               # sum_i (v_i^T x_t) u_i
                y = y + torch.dot(vi, x) * ui
        else:
            self.l += 1
            g = torch.as_tensor(philox.gaussian_vector(self.seed, self.trial, t, self.n,
                                                       self.r, self.sigma))
            p = apply_in_order(self.L, x)                    # L_{l-1} ... L_1 x_t
            self.L.append(Reflector(self.l - 1, p))          # L_l = H_l(p)
            u = apply_reversed(self.L, unit(self.m, self.l - 1))  # L_1 ... L_l e_l
            v = apply_reversed(self.R, g)                    # R_1 ... R_r Z_{1:r} g_t
            self.u.append(u)
            self.v.append(v)
            y = torch.zeros(self.n, dtype=F64)
            for ui, vi in zip(self.u, self.v):               # sum_i (u_i^T x_t) v_i
                y = y + torch.dot(ui, x) * vi
        self.qstep.append(not transpose)
        self.t = t
        return y

    def revealed(self):
        """sum_i u_i v_i^T (m x n, small cases only); the part of Q^(t) built so far (eq. Gaussian_t)."""
        Q = torch.zeros(self.m, self.n, dtype=F64)
        for ui, vi in zip(self.u, self.v):
            Q = Q + torch.outer(ui, vi)
        return Q

    def probe(self, x, transpose=False):
        """Q^(t) x (or Q^(t)^T x) from the revealed part, without adding a step.

        Returns (y, unrevealed): unrevealed is ||Z_{1:r} R_r...R_1 x|| for Q (resp. with L
        and l for Q^T); the hidden Gaussian block of eq. (Gaussian_t) is invisible to x
        exactly when it is zero.
        """
        x = _vec(x)
        if not transpose:
            q = apply_in_order(self.R, x)
            unrevealed = torch.sqrt(torch.dot(q[self.r:], q[self.r:]))
            y = torch.zeros(self.m, dtype=F64)
            for ui, vi in zip(self.u, self.v):
                y = y + torch.dot(vi, x) * ui
        else:
            q = apply_in_order(self.L, x)
            unrevealed = torch.sqrt(torch.dot(q[self.l:], q[self.l:]))
            y = torch.zeros(self.n, dtype=F64)
            for ui, vi in zip(self.u, self.v):
                y = y + torch.dot(ui, x) * vi
        return y, unrevealed


def make_oracle(ensemble, m, n, T_max, seed, trial=0, sigma=1.0):
    if ensemble == "haar":
        if m != n:
            raise ValueError("Haar requires m == n")
        return HaarOracle(n, T_max, seed, trial)
    if ensemble == "ginibre":
        return GinibreOracle(m, n, T_max, seed, trial, sigma)
    raise ValueError(ensemble)
