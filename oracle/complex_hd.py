"""Complex Householder Dice: the unitary group, complex Ginibre and GUE (test infrastructure only).

The paper's section "Other Random Matrix Ensembles" states that the construction carries over
to complex matrices, with M^T replaced by M^H, and gives the complex reflector of
eq. (Householder_c): for v in C^n with v_1/||v|| = r e^{i theta} (theta = 0 when v_1 = 0),

    H(v) = -e^{-i theta} [ I - (v/||v|| + e^{i theta} e_1)(v/||v|| + e^{i theta} e_1)^H / (1 + r) ],

unitary, with H(v) v = ||v|| e_1 and H(v)^H e_1 = v/||v||.  It is not Hermitian, so the real
Algorithm 2 is restated with adjoints where a reflector acts from the left of the revealed
block.  Q = L_1^H ... L_t^H [I_t 0; 0 Q~] R_t ... R_1 with Q~ ~ Haar(U(n - t)):

  * Q step:   p = R_{t-1} ... R_1 x,  R_t = H_t(p),  L_t = H_t(g_t),
              y = L_1^H ... L_t^H R_t p   (R_t p = [p_head; alpha; 0], alpha = ||p[t:]||);
  * Q^H step: p = L_{t-1} ... L_1 x,  L_t = H_t(p),  R_t = H_t(g_t),
              y = R_1^H ... R_t^H L_t p.

H_k(p) is the identity on the first k coordinates and H(p[k:]) on the rest (eq.
Householder_e), the identity when p[k:] = 0.  In the real case H^H = H^T = H and this is
Algorithm 2.

Complex Ginibre CGin(m, n) (entries sigma CN(0, 1)): Algorithm 1 with the same adjoints.  Its
revealed part is sum_i u_i v_i^H, and the hidden block sits between L^H and R (Q = L_1^H ...
L_l^H [revealed; 0 G~] R_r ... R_1):

  * Q step:   r <- r + 1, g in C^m drawn on rows l..m-1 (Z_{1:l} g), p = R_{r-1} ... R_1 x,
              R_r = H_r(p), u_t = L_1^H ... L_l^H (Z g), v_t = R_1^H ... R_r^H e_r,
              y = sum_{i <= t} (v_i^H x) u_i;
  * Q^H step: l <- l + 1, g in C^n drawn on rows r..n-1, L_l = H_l(L_{l-1} ... L_1 x),
              u_t = L_1^H ... L_l^H e_l, v_t = R_1^H ... R_r^H (Z g), y = sum_i (u_i^H x) v_i.

GUE(n) = (Q + Q^H) / sqrt(2) for Q ~ CGin(n, n) (two products of one square state per query).

Complex draws: entry i of step t's vector g_t is (N_{2i} + i N_{2i+1}) / sqrt(2), with N_j
the j-th normal of step t's Philox stream (the pair that one Box-Muller transform gives), so
g_t ~ CN(0, I); masked entries i < first are zero and never drawn.
"""
import math

import numpy as np
import torch

from . import philox

C128 = torch.complex128


def _cvec(x):
    if isinstance(x, torch.Tensor):
        return x.to(C128)
    return torch.as_tensor(np.asarray(x, dtype=np.complex128))


def complex_gaussian_vector(seed, trial, step, dim, first):
    """g in C^dim, entries CN(0, 1) at 0-based indices first..dim-1, zeros before."""
    g = np.zeros(dim, dtype=np.complex128)
    if first < dim:
        nrm = philox.normals(seed, trial, step, 2 * first, 2 * (dim - first))
        g[first:] = (nrm[0::2] + 1j * nrm[1::2]) / math.sqrt(2.0)
    return g


class ComplexReflector:
    """H_{k+1}(p) of eq. (Householder_c) on the coordinates k.. (identity on the first k)."""

    def __init__(self, k, p):
        p = _cvec(p)
        a = p[k:]
        self.k = k
        self.alpha = torch.linalg.vector_norm(a)
        self.identity = bool(self.alpha == 0)
        if self.identity:
            return
        v1 = a[0] / self.alpha
        self.r = torch.abs(v1)
        self.phase = (v1 / self.r) if float(self.r) > 0 else torch.tensor(1.0 + 0j, dtype=C128)  # e^{i theta}
        e1 = torch.zeros_like(a)
        e1[0] = 1.0
        self.w = a / self.alpha + self.phase * e1
        self.scale = -torch.conj(self.phase)                                         # -e^{-i theta}

    def apply(self, z):
        """H z (z not modified)."""
        z = _cvec(z)
        if self.identity:
            return z.clone()
        seg = z[self.k:]
        seg = self.scale * (seg - self.w * (torch.vdot(self.w, seg) / (1.0 + self.r)))
        return torch.cat([z[:self.k], seg])

    def apply_h(self, z):
        """H^H z."""
        z = _cvec(z)
        if self.identity:
            return z.clone()
        seg = torch.conj(self.scale) * z[self.k:]
        seg = seg - self.w * (torch.vdot(self.w, seg) / (1.0 + self.r))
        return torch.cat([z[:self.k], seg])

    def dense(self, dim):
        eye = torch.eye(dim, dtype=C128)
        return torch.stack([self.apply(eye[:, j]) for j in range(dim)], dim=1)


def unit(dim, k):
    e = torch.zeros(dim, dtype=C128)
    e[k] = 1.0
    return e


class ComplexHaarOracle:
    """Householder Dice for Q ~ Haar(U(n)): y_t = M_t x_t with M_t in {Q, Q^H}."""

    def __init__(self, n, T_max, seed, trial=0):
        if T_max > n:
            raise ValueError("requires T <= n")
        self.n, self.T_max, self.seed, self.trial = n, T_max, seed, trial
        self.R, self.L, self.t = [], [], 0

    def apply(self, x, adjoint=False):
        t = self.t + 1
        if t > self.T_max:
            raise ValueError("step would exceed T_max")
        x = _cvec(x)
        g = complex_gaussian_vector(self.seed, self.trial, t, self.n, t - 1)
        if not adjoint:
            p = x
            for h in self.R:
                p = h.apply(p)                           # R_{t-1} ... R_1 x
            Rt, Lt = ComplexReflector(t - 1, p), ComplexReflector(t - 1, g)
            self.R.append(Rt)
            self.L.append(Lt)
            y = Rt.apply(p)
            for h in reversed(self.L):
                y = h.apply_h(y)                         # L_1^H ... L_t^H
        else:
            p = x
            for h in self.L:
                p = h.apply(p)                           # L_{t-1} ... L_1 x
            Lt, Rt = ComplexReflector(t - 1, p), ComplexReflector(t - 1, g)
            self.L.append(Lt)
            self.R.append(Rt)
            y = Lt.apply(p)
            for h in reversed(self.R):
                y = h.apply_h(y)                         # R_1^H ... R_t^H
        self.t = t
        return y

    def matrix(self):
        """The implied Q once t = n (nothing unrevealed): L_1^H ... L_n^H R_n ... R_1."""
        if self.t != self.n:
            raise ValueError("Q is determined only at t = n")
        eye = torch.eye(self.n, dtype=C128)
        cols = []
        for j in range(self.n):
            z = eye[:, j]
            for h in self.R:
                z = h.apply(z)
            for h in reversed(self.L):
                z = h.apply_h(z)
            cols.append(z)
        return torch.stack(cols, dim=1)


def apply_h_reversed(refls, z):
    """refls[0]^H refls[1]^H ... refls[-1]^H z (the last reflector acts first)."""
    for h in reversed(refls):
        z = h.apply_h(z)
    return z


class ComplexGinibreOracle:
    """Algorithm 1 on complex matrices: y_t = M_t x_t, M_t in {Q, Q^H}, Q ~ CGin(m, n) with
    entries sigma CN(0, 1), one reflector at a time, in the paper's order."""

    def __init__(self, m, n, T_max, seed, trial=0, sigma=1.0):
        if T_max > min(m, n):
            raise ValueError("Algorithm 1 requires T <= min(m, n)")
        self.m, self.n, self.T_max = m, n, T_max
        self.seed, self.trial, self.sigma = seed, trial, sigma
        self.R, self.L, self.u, self.v = [], [], [], []
        self.t = self.r = self.l = 0

    def apply(self, x, adjoint=False):
        t = self.t + 1
        if t > self.T_max:
            raise ValueError("step would exceed T_max")
        x = _cvec(x)
        if not adjoint:
            self.r += 1
            g = self.sigma * torch.as_tensor(complex_gaussian_vector(self.seed, self.trial, t, self.m, self.l))
            p = x
            for h in self.R:
                p = h.apply(p)                                   # R_{r-1} ... R_1 x
            self.R.append(ComplexReflector(self.r - 1, p))       # R_r = H_r(p)
            self.u.append(apply_h_reversed(self.L, g))           # L_1^H ... L_l^H Z g
            self.v.append(apply_h_reversed(self.R, unit(self.n, self.r - 1)))   # R_1^H ... R_r^H e_r
            y = torch.zeros(self.m, dtype=C128)
            for ui, vi in zip(self.u, self.v):                   # sum_i (v_i^H x) u_i
                y = y + torch.vdot(vi, x) * ui
        else:
            self.l += 1
            g = self.sigma * torch.as_tensor(complex_gaussian_vector(self.seed, self.trial, t, self.n, self.r))
            q = x
            for h in self.L:
                q = h.apply(q)                                   # L_{l-1} ... L_1 x
            self.L.append(ComplexReflector(self.l - 1, q))       # L_l = H_l(q)
            self.u.append(apply_h_reversed(self.L, unit(self.m, self.l - 1)))   # L_1^H ... L_l^H e_l
            self.v.append(apply_h_reversed(self.R, g))           # R_1^H ... R_r^H Z g
            y = torch.zeros(self.n, dtype=C128)
            for ui, vi in zip(self.u, self.v):                   # sum_i (u_i^H x) v_i
                y = y + torch.vdot(ui, x) * vi
        self.t = t
        return y

    def revealed(self):
        """sum_i u_i v_i^H (m x n): the part of Q built so far (the whole Q once all of it is
        revealed)."""
        Q = torch.zeros(self.m, self.n, dtype=C128)
        for ui, vi in zip(self.u, self.v):
            Q = Q + torch.outer(ui, vi.conj())
        return Q


def gue_apply(gin, x):
    """W x for W = (Q + Q^H) / sqrt(2) ~ GUE(n): a Q and a Q^H product of one square complex
    Ginibre state."""
    x = _cvec(x)
    return (gin.apply(x, False) + gin.apply(x, True)) / math.sqrt(2.0)
