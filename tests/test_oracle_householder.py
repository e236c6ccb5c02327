"""Pins for the oracle's reflector (oracle/hd.py: Reflector).

* eq. (Householder_property): H(v) e_1 = v/||v|| and H(v) v = ||v|| e_1; H symmetric and
  orthogonal (Section 3.1) -- for v_1 > 0, v_1 < 0 and v_1 = 0.  The sign rule read as
  +1/-1 is what makes H orthogonal; with "0 otherwise" H would be 0 for v_1 < 0.
* eq. (ortho): Z_{1:k} H_k(p) p = 0, and H_k(p) = I when p[k:n] = 0 (eq. Householder_e).
* The complex reflector of eq. (Householder_c) restricted to real v equals H(v)
  (stated after that equation); the formula is evaluated here as a dense matrix.
* Applying H_r(R_{r-1}...R_1 x_r) column by column is Householder QR (Remark after
  Algorithm 1): the result is upper triangular and matches LAPACK's R up to row signs.
"""
import numpy as np
import pytest
import torch

from oracle.hd import Reflector, apply_in_order


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


@pytest.mark.parametrize("first", [1.3, -0.7, 0.0])
def test_householder_property(first):
    n = 9
    v = _rand(n, 1)
    v[0] = first
    H = Reflector(0, v).dense(n).numpy()
    nv = np.linalg.norm(v)
    e1 = np.eye(n)[:, 0]
    np.testing.assert_allclose(H, H.T, atol=1e-15)
    np.testing.assert_allclose(H.T @ H, np.eye(n), atol=1e-14)
    np.testing.assert_allclose(H @ e1, v / nv, atol=1e-15)
    np.testing.assert_allclose(H @ v, nv * e1, atol=1e-14)
    # eigenvalues +-1 (Section 3.1)
    ev = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(np.abs(ev), 1.0, atol=1e-13)


def test_generalised_reflector_zeroes_tail():
    n = 11
    p = _rand(n, 2)
    for k in range(n):
        Hp = Reflector(k, p).apply(p).numpy()
        np.testing.assert_array_equal(Hp[:k], p[:k])          # I_{k-1} block
        assert abs(Hp[k] - np.linalg.norm(p[k:])) < 1e-14     # ||p[k:n]|| e_k
        np.testing.assert_allclose(Hp[k + 1:], 0.0, atol=1e-14)  # Z_{1:k} H_k(p) p = 0


def test_zero_tail_gives_identity():
    n = 6
    p = np.array([1.0, -2.0, 0.0, 0.0, 0.0, 0.0])
    h = Reflector(2, p)
    assert h.identity
    w = _rand(n, 3)
    np.testing.assert_array_equal(h.apply(w).numpy(), w)


def test_complex_reflector_reduces_to_real():
    n = 7
    for first in (0.9, -0.4, 0.0):
        v = _rand(n, 4).astype(np.complex128)
        v[0] = first
        nv = np.linalg.norm(v)
        r = abs(v[0]) / nv
        theta = 0.0 if v[0] == 0 else np.angle(v[0] / nv)
        w = v / nv + np.exp(1j * theta) * np.eye(n)[:, 0]
        Hc = -np.exp(-1j * theta) * (np.eye(n) - np.outer(w, w.conj()) / (1.0 + r))
        H = Reflector(0, v.real).dense(n).numpy()
        np.testing.assert_allclose(Hc.imag, 0.0, atol=1e-15)
        np.testing.assert_allclose(Hc.real, H, atol=1e-14)


def test_sequential_reflectors_are_householder_qr():
    m, k = 8, 5
    X = np.random.default_rng(5).standard_normal((m, k))
    refl = []
    for j in range(k):
        p = apply_in_order(refl, X[:, j])
        refl.append(Reflector(j, p))
    Rt = np.stack([apply_in_order(refl, X[:, j]).numpy() for j in range(k)], axis=1)
    np.testing.assert_allclose(np.tril(Rt, -1), 0.0, atol=1e-13)
    R_lapack = np.linalg.qr(X, mode="r")
    np.testing.assert_allclose(np.abs(Rt[:k]), np.abs(R_lapack), rtol=1e-12, atol=1e-13)
    # the diagonal is ||p[k:n]|| >= 0 (H v = ||v|| e_1), unlike LAPACK's sign choice
    assert np.all(np.diag(Rt[:k]) >= 0)


def test_reflector_is_differentiable():
    p = torch.tensor(_rand(5, 6), requires_grad=True)
    w = torch.tensor(_rand(5, 7))
    out = Reflector(1, p).apply(w).sum()
    out.backward()
    assert p.grad is not None and torch.isfinite(p.grad).all()
