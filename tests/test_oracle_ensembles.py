"""Pins of the ensemble compositions (paper, section "Other Random Matrix Ensembles"), on
the oracle:

* GOE: W = (Q + Q^T)/sqrt(2) has W_ii ~ N(0, 2) and W_ij ~ N(0, 1) (i != j): KS tests over
  independent states; the revealed block of W is symmetric (the two products of every query
  come from one Q).
* Q = U Sigma V (eq. inv): reconstructed from column (or row) queries at small sizes, its
  singular values are s exactly (U, V orthogonal), square and rectangular; with s = 1 it
  keeps norms.
"""
import math

import numpy as np
import pytest
import torch
from scipy import stats

from oracle.ensembles import goe_apply, make_goe, make_usv, usv_apply


def e(n, i):
    v = torch.zeros(n, dtype=torch.float64)
    v[i] = 1.0
    return v


def test_goe_entry_laws():
    n, trials = 12, 2000
    diag, off = [], []
    for s in range(trials):
        g = make_goe(n, 2, seed=1000 + s)
        w1 = goe_apply(g, e(n, 0)).numpy()
        diag.append(w1[0])
        off.append(w1[3])
    assert stats.kstest(np.array(diag) / math.sqrt(2.0), "norm").pvalue > 1e-3
    assert stats.kstest(np.array(off), "norm").pvalue > 1e-3
    # a missing 1/sqrt(2) would give variance 4 and 2
    assert abs(np.var(diag) - 2.0) < 0.25 and abs(np.var(off) - 1.0) < 0.15


def test_goe_revealed_block_is_symmetric():
    n, q = 14, 7
    g = make_goe(n, 2 * q, seed=5)
    cols = [goe_apply(g, e(n, j)).numpy() for j in range(q)]
    W = np.stack(cols, axis=1)[:q, :]          # W[:q, :q]
    assert np.abs(W - W.T).max() <= 1e-13 * np.abs(W).max()


@pytest.mark.parametrize("m,n", [(8, 8), (6, 9), (9, 6)])
def test_usv_singular_values(m, n):
    rng = np.random.default_rng(m * 10 + n)
    k = min(m, n)
    s = np.sort(rng.uniform(0.5, 3.0, k))[::-1].copy()
    U, V = make_usv(m, n, min(m, n), seed_u=3, seed_v=4)
    if m <= n:   # rows: Q^T e_i, i < m (one product of each state per query)
        Qt = np.stack([usv_apply(U, V, s, e(m, i), transpose=True).numpy() for i in range(m)], axis=1)
        sv = np.linalg.svd(Qt, compute_uv=False)
    else:        # columns: Q e_j, j < n
        Q = np.stack([usv_apply(U, V, s, e(n, j)).numpy() for j in range(n)], axis=1)
        sv = np.linalg.svd(Q, compute_uv=False)
    np.testing.assert_allclose(np.sort(sv)[::-1][:k], s, rtol=1e-12)


def test_usv_unit_sigma_keeps_norms():
    n = 50
    U, V = make_usv(n, n, 10, seed_u=7, seed_v=8)
    rng = np.random.default_rng(0)
    for t in range(10):
        x = torch.tensor(rng.standard_normal(n))
        y = usv_apply(U, V, np.ones(n), x, transpose=bool(t % 2))
        assert abs(y.norm().item() / x.norm().item() - 1.0) <= 1e-13
