"""Pins of the complex Householder Dice oracle (Haar measure on the unitary group; the
paper's section "Other Random Matrix Ensembles", eq. Householder_c):

* the complex reflector is unitary, maps v to ||v|| e_1, its adjoint maps e_1 to v/||v||, and
  for real v it is the real reflector of eq. Householder;
* step 1 gives y_1 = ||x_1|| g_1/||g_1|| for Q and for Q^H;
* every product keeps norms; at n = 6, T = n the implied Q is unitary and reproduces every
  earlier query (brute force);
* law: |Q_11|^2 ~ Beta(1, n - 1), arg Q_11 uniform, |Q_11|^2 + |Q_12|^2 ~ Beta(2, n - 2)
  (the first row of a Haar unitary matrix is uniform on the complex sphere).
"""
import math

import numpy as np
import pytest
import torch
from scipy import stats

from oracle.complex_hd import ComplexHaarOracle, ComplexReflector, complex_gaussian_vector, unit
from oracle.hd import Reflector


def crand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("n,seed", [(1, 1), (5, 2), (17, 3)])
def test_complex_reflector_identities(n, seed):
    v = torch.tensor(crand(n, seed))
    H = ComplexReflector(0, v).dense(n)
    eye = torch.eye(n, dtype=torch.complex128)
    assert torch.linalg.matrix_norm(H.conj().T @ H - eye) <= 1e-13
    nv = torch.linalg.vector_norm(v)
    assert torch.linalg.vector_norm(H @ v - nv * unit(n, 0)) <= 1e-13 * nv
    assert torch.linalg.vector_norm(H.conj().T @ unit(n, 0) - v / nv) <= 1e-13


def test_complex_reflector_reduces_to_real_and_handles_zero_pivot():
    n = 9
    v = np.random.default_rng(4).standard_normal(n)
    for vv in (v, -v, np.concatenate([[0.0], v[1:]])):
        Hc = ComplexReflector(0, vv).dense(n)
        Hr = Reflector(0, torch.tensor(vv)).dense(n)
        assert torch.linalg.matrix_norm(Hc - Hr.to(torch.complex128)) <= 1e-13
    ident = ComplexReflector(3, np.concatenate([crand(3, 5), np.zeros(4)]))
    z = torch.tensor(crand(7, 6))
    assert torch.equal(ident.apply(z), z)


@pytest.mark.parametrize("adjoint", [False, True])
def test_first_step_closed_form(adjoint):
    n, seed = 11, 7
    x = crand(n, 8)
    y = ComplexHaarOracle(n, 3, seed).apply(x, adjoint).numpy()
    g = complex_gaussian_vector(seed, 0, 1, n, 0)
    np.testing.assert_allclose(y, np.linalg.norm(x) * g / np.linalg.norm(g), rtol=0, atol=1e-13 * np.linalg.norm(x))


def test_norms_kept_and_brute_force_reconstruction():
    n = 6
    o = ComplexHaarOracle(n, n, 9)
    sched = [False, True, True, False, True, False]
    xs, ys = [], []
    for t in range(n):
        x = crand(n, 20 + t)
        y = o.apply(x, sched[t]).numpy()
        assert abs(np.linalg.norm(y) / np.linalg.norm(x) - 1.0) <= 1e-13
        xs.append(x)
        ys.append(y)
    Q = o.matrix().numpy()
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 1e-13
    for t in range(n):
        M = Q.conj().T if sched[t] else Q
        np.testing.assert_allclose(M @ xs[t], ys[t], rtol=0, atol=1e-12)


def test_first_row_law():
    n, trials = 5, 2000
    a11, a12, ph = [], [], []
    for s in range(trials):
        o = ComplexHaarOracle(n, 2, 100 + s)
        c1 = o.apply(unit(n, 0)).numpy()       # column 1: Q_11 = c1[0]
        c2 = o.apply(unit(n, 1)).numpy()       # column 2: Q_12 = c2[0]
        a11.append(abs(c1[0]) ** 2)
        a12.append(abs(c1[0]) ** 2 + abs(c2[0]) ** 2)
        ph.append(np.angle(c1[0]))
    assert stats.kstest(a11, stats.beta(1, n - 1).cdf).pvalue > 1e-3
    assert stats.kstest(a12, stats.beta(2, n - 2).cdf).pvalue > 1e-3
    assert stats.kstest(ph, stats.uniform(-math.pi, 2 * math.pi).cdf).pvalue > 1e-3


def test_revealed_unitary_trace_moments():
    """The fully revealed Q at n = 6 against the trace moments of the Haar measure on U(n)
    (Diaconis and Shahshahani, 1994): for sum_j j a_j <= n, E prod_j |tr Q^j|^{2 a_j} =
    prod_j j^{a_j} a_j!, and E (tr Q)^2 = E tr Q = 0.  So E |tr Q|^2 = 1, E |tr Q|^4 = 2,
    E |tr Q|^6 = 6 and E |tr Q^2|^2 = 2.  The queries mix Q and Q^H steps, so both reflector
    stacks and their adjoints enter the reconstruction.  The queries are the same fixed
    vectors in every trial, so all the randomness is the draws'; Theorem 2's complex analogue
    says Q is Haar for any queries independent of it.  (A planted mistake with real draws
    still passed these moments at this sample size, so the law of the draws themselves is
    left to the uniform phase in test_first_row_law.)"""
    n, trials = 6, 600
    sched = [False, True, True, False, True, False]
    rng = np.random.default_rng(3)
    queries = [rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(n)]
    t1, t2 = [], []
    for i in range(trials):
        o = ComplexHaarOracle(n, n, 500, trial=i)
        for t in range(n):
            o.apply(queries[t], sched[t])
        Q = o.matrix().numpy()
        t1.append(np.trace(Q))
        t2.append(np.trace(Q @ Q))
    t1, t2 = np.array(t1), np.array(t2)
    a1 = np.abs(t1) ** 2
    for sample, want in ((t1.real, 0.0), (t1.imag, 0.0), ((t1 ** 2).real, 0.0), (a1, 1.0),
                         (a1 ** 2, 2.0), (a1 ** 3, 6.0), (np.abs(t2) ** 2, 2.0)):
        se = sample.std(ddof=1) / np.sqrt(trials)
        assert abs(sample.mean() - want) <= 4.5 * se, (sample.mean(), want, se)


# ---- complex Ginibre (Algorithm 1 with adjoints) and GUE ------------------------------------
from oracle.complex_hd import ComplexGinibreOracle, gue_apply   # noqa: E402


@pytest.mark.parametrize("adjoint", [False, True])
def test_complex_ginibre_first_step_closed_form(adjoint):
    """Step 1: v_1 = x / ||x|| (R_1^H e_1 = x/||x||), u_1 = g, so y_1 = ||x|| g (sigma g)."""
    m, n, seed, sigma = 7, 11, 3, 0.5
    x = crand(m if adjoint else n, 4)
    y = ComplexGinibreOracle(m, n, 3, seed, sigma=sigma).apply(x, adjoint).numpy()
    g = sigma * complex_gaussian_vector(seed, 0, 1, n if adjoint else m, 0)
    np.testing.assert_allclose(y, np.linalg.norm(x) * g, rtol=0, atol=1e-13 * np.linalg.norm(x))


@pytest.mark.parametrize("m,n", [(6, 6), (5, 8), (8, 5)])
def test_complex_ginibre_revealed_part_reproduces_queries(m, n):
    """Every earlier query is reproduced by the revealed part sum_i u_i v_i^H (its hidden
    block never meets an earlier input), for mixed Q / Q^H schedules, rectangular both ways."""
    T = min(m, n)
    sched = [t % 3 == 1 for t in range(T)]
    o = ComplexGinibreOracle(m, n, T, 21)
    qs, ys = [], []
    for t in range(T):
        x = crand(m if sched[t] else n, 30 + t)
        ys.append(o.apply(x, sched[t]).numpy())
        qs.append(x)
    Q = o.revealed().numpy()
    for t in range(T):
        M = Q.conj().T if sched[t] else Q
        np.testing.assert_allclose(M @ qs[t], ys[t], rtol=0, atol=1e-12 * max(1.0, np.linalg.norm(ys[t])))


def test_complex_ginibre_all_q_square_reconstruction_has_complex_gaussian_entries():
    """Square, all Q, T = n: the revealed part is all of Q.  Over independent trials its
    entries are CN(0, sigma^2): real and imaginary parts N(0, sigma^2 / 2) (KS), uncorrelated,
    and E Q_ij^2 = 0 (circular symmetry: a planted real draw makes E Q^2 = sigma^2)."""
    n, trials, sigma = 4, 800, 1.5
    rng = np.random.default_rng(9)
    qs = [rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(n)]
    ent = []
    for i in range(trials):
        o = ComplexGinibreOracle(n, n, n, 77, trial=i, sigma=sigma)
        for t in range(n):
            o.apply(qs[t], False)
        ent.append(o.revealed().numpy().reshape(-1))
    ent = np.array(ent)
    sd = sigma / math.sqrt(2.0)
    for j in (0, 5, 15):
        assert stats.kstest(ent[:, j].real / sd, "norm").pvalue > 1e-3
        assert stats.kstest(ent[:, j].imag / sd, "norm").pvalue > 1e-3
        sq = ent[:, j] ** 2
        se = np.abs(sq).std(ddof=1) / math.sqrt(trials)
        assert abs(sq.mean()) <= 4.5 * se, (j, sq.mean(), se)


def test_gue_entry_laws_and_hermitian_revealed_block():
    """W = (Q + Q^H)/sqrt(2): W_11 ~ N(0, sigma^2) real, W_12 ~ CN(0, sigma^2); and every
    query pair W e_j, W e_k is consistent with a Hermitian W: e_k^H W e_j = conj(e_j^H W e_k)."""
    n, trials = 5, 1500
    w11, w12, herm = [], [], []
    for i in range(trials):
        o = ComplexGinibreOracle(n, n, 4, 5, trial=i)
        c1 = gue_apply(o, unit(n, 0)).numpy()
        c2 = gue_apply(o, unit(n, 1)).numpy()
        w11.append(c1[0])
        w12.append(c2[0])
        herm.append(abs(c2[0] - np.conj(c1[1])))
    w11, w12 = np.array(w11), np.array(w12)
    assert np.abs(w11.imag).max() <= 1e-13
    assert stats.kstest(w11.real, "norm").pvalue > 1e-3
    assert stats.kstest(w12.real * math.sqrt(2.0), "norm").pvalue > 1e-3
    assert stats.kstest(w12.imag * math.sqrt(2.0), "norm").pvalue > 1e-3
    assert max(herm) <= 1e-12
