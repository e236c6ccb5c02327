"""Pins for the oracle's Algorithms 1 and 2 (oracle/hd.py).

Haar (Algorithm 2, Section 3.3):
  * step 1 closed form Q x_1 = ||x_1|| g_1 / ||g_1||  (after eq. H_1);
  * ||y_t|| = ||x_t|| at every step (Q orthogonal);
  * consistency: the state after s steps reproduces every earlier query, and Q^T applied
    to an earlier output returns the earlier input (claim (b) of Theorem 2 and the
    sparsity of R_t...R_1 x_t noted after eq. H_2);
  * brute force at n = 8, T = n: L_1..L_n R_n..R_1 is the whole Q (eq. H_t with t = n);
    it is orthogonal and reproduces all queries.
Ginibre (Algorithm 1, Section 3.2):
  * step 1 closed form Q x_1 = ||x_1|| g_1  (after eq. Gaussian_1), scaled by sigma;
  * step 2 closed form Q x_2 = (v_1^T x_2) u_1 + (v_2^T x_2) u_2 with u_1 = g_1, u_2 = g_2,
    v_1 = R_1 e_1 = x_1/||x_1||, v_2 = R_1 R_2 e_2 (eq. Gaussian_2);
  * v_i^T x_t = (R_r...R_1 x_t)[r_i] for Q-steps i (v_i = R_1...R_r e_{r_i});
  * square, all-Q, T = n: sum_i u_i v_i^T is the whole Q and reproduces all queries;
    mixed schedules reproduce all queries through the revealed part;
  * the v_i of Q-steps (and the u_i of Q^T-steps) are orthonormal.
"""
import numpy as np
import pytest
import torch

from oracle import philox
from oracle.dynamics import f_sign_mem, f_tanh, run, schedule_alternating
from oracle.hd import GinibreOracle, HaarOracle, apply_in_order

rng = np.random.default_rng


def test_haar_first_step_closed_form():
    n = 50
    x = rng(1).standard_normal(n)
    st = HaarOracle(n, 5, seed=42)
    y = st.apply(x).numpy()
    g = philox.normals(42, 0, 1, 0, n)
    np.testing.assert_allclose(y, np.linalg.norm(x) * g / np.linalg.norm(g), rtol=0, atol=1e-14)


def test_haar_first_step_transpose_closed_form():
    n = 30
    x = rng(2).standard_normal(n)
    st = HaarOracle(n, 5, seed=3)
    y = st.apply(x, transpose=True).numpy()
    g = philox.normals(3, 0, 1, 0, n)
    np.testing.assert_allclose(y, np.linalg.norm(x) * g / np.linalg.norm(g), atol=1e-14)


@pytest.mark.parametrize("sched", ["alt", "allq", "mixed"])
def test_haar_norm_and_consistency(sched):
    n, T = 64, 20
    pattern = {"alt": lambda t: t % 2 == 0, "allq": lambda t: False,
               "mixed": lambda t: t in (2, 3, 7, 11, 12, 13)}[sched]
    st = HaarOracle(n, T, seed=9)
    xs, ys = run(st, rng(3).standard_normal(n), T, f_sign_mem, pattern)
    for t in range(1, T + 1):
        x, y = xs[t - 1], ys[t - 1]
        assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-13 * np.linalg.norm(x)
    for t in range(1, T + 1):
        tr = pattern(t)
        yp, unrev = st.probe(xs[t - 1], transpose=tr)
        assert float(unrev) < 1e-12 * np.linalg.norm(xs[t - 1])
        np.testing.assert_allclose(yp.numpy(), ys[t - 1], atol=1e-12 * np.linalg.norm(ys[t - 1]))
        xb, unrev2 = st.probe(ys[t - 1], transpose=not tr)
        assert float(unrev2) < 1e-12 * np.linalg.norm(ys[t - 1])
        np.testing.assert_allclose(xb.numpy(), xs[t - 1], atol=1e-12 * np.linalg.norm(xs[t - 1]))


def test_haar_brute_force_n8():
    n = 8
    pattern = lambda t: t in (2, 5, 6)
    st = HaarOracle(n, n, seed=5)
    xs, ys = run(st, rng(4).standard_normal(n), n, f_sign_mem, pattern)
    Q = st.dense().numpy()
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-14)
    for t in range(1, n + 1):
        M = Q.T if pattern(t) else Q
        np.testing.assert_allclose(M @ xs[t - 1], ys[t - 1], atol=1e-13)


def test_haar_probe_of_fresh_vector_reports_unrevealed_part():
    n = 20
    st = HaarOracle(n, 5, seed=1)
    st.apply(rng(5).standard_normal(n))
    _, unrev = st.probe(rng(6).standard_normal(n))
    assert float(unrev) > 0.5


def test_ginibre_first_step_closed_form():
    m, n, sigma = 40, 30, 0.25
    x = rng(7).standard_normal(n)
    st = GinibreOracle(m, n, 5, seed=8, sigma=sigma)
    y = st.apply(x).numpy()
    g = sigma * philox.normals(8, 0, 1, 0, m)
    np.testing.assert_allclose(y, np.linalg.norm(x) * g, atol=1e-14)


def test_ginibre_second_step_closed_form():
    m, n = 12, 9
    x1, x2 = rng(8).standard_normal(n), rng(9).standard_normal(n)
    st = GinibreOracle(m, n, 5, seed=10)
    st.apply(x1)
    y2 = st.apply(x2).numpy()
    g1 = philox.normals(10, 0, 1, 0, m)
    g2 = philox.normals(10, 0, 2, 0, m)
    v1 = x1 / np.linalg.norm(x1)               # R_1 e_1 = x_1/||x_1||
    # v_2 = R_1 R_2 e_2: R_1 is H(x_1); R_2 = H_2(R_1 x_2), R_2 e_2 = (R_1 x_2)[2:]/norm
    R1 = st.R[0].dense(n).numpy()
    p = R1 @ x2
    w = np.zeros(n)
    w[1:] = p[1:] / np.linalg.norm(p[1:])
    v2 = R1 @ w
    np.testing.assert_allclose(y2, (v1 @ x2) * g1 + (v2 @ x2) * g2, atol=1e-13)


def test_ginibre_coefficients_come_from_p():
    m, n, T = 15, 25, 8
    pattern = lambda t: t in (3, 4, 6)
    st = GinibreOracle(m, n, T, seed=11)
    for t in range(1, T + 1):
        st.apply(rng(200 + t).standard_normal(m if pattern(t) else n), transpose=pattern(t))
    # at the end, r = #Q-steps; for each Q-step i with pivot r_i, v_i = R_1..R_r e_{r_i}
    x = rng(11).standard_normal(n)
    q = apply_in_order(st.R, x).numpy()
    ri = 0
    for i, isq in enumerate(st.qstep):
        if isq:
            assert abs(float(torch.dot(st.v[i], torch.as_tensor(x))) - q[ri]) < 1e-13
            ri += 1


def test_ginibre_square_all_q_reconstruction():
    n = 7
    st = GinibreOracle(n, n, n, seed=12)
    xs, ys = run(st, rng(12).standard_normal(n), n, f_tanh, lambda t: False)
    Q = st.revealed().numpy()
    for t in range(1, n + 1):
        np.testing.assert_allclose(Q @ xs[t - 1], ys[t - 1], atol=1e-13)
    # Q v_i = u_i for the orthonormal v_i of the Q-steps (basis structure of eq. Gaussian_t)
    V = torch.stack(st.v, 1).numpy()
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-14)


@pytest.mark.parametrize("m,n", [(9, 13), (13, 9)])
def test_ginibre_mixed_schedule_consistency(m, n):
    T = 8
    pattern = lambda t: t % 3 == 0
    st = GinibreOracle(m, n, T, seed=13, sigma=0.5)
    x1 = rng(13).standard_normal(n)
    # alternate dimensions: Q maps R^n -> R^m, Q^T maps R^m -> R^n
    xs, ys, x = [], [], x1
    for t in range(1, T + 1):
        tr = pattern(t)
        y = st.apply(x, transpose=tr).numpy()
        xs.append(x)
        ys.append(y)
        nxt_dim = n if not pattern(t + 1) else m
        # next input must live where M_{t+1} acts: keep the output if dims fit, else draw
        x = np.tanh(y) if y.shape[0] == nxt_dim else rng(100 + t).standard_normal(nxt_dim)
    Qrev = st.revealed().numpy()
    for t in range(1, T + 1):
        M = Qrev.T if pattern(t) else Qrev
        np.testing.assert_allclose(M @ xs[t - 1], ys[t - 1], atol=1e-12)
        yp, unrev = st.probe(xs[t - 1], transpose=pattern(t))
        assert float(unrev) < 1e-12
    # Q-step v's orthonormal, Q^T-step u's orthonormal
    Vq = np.stack([st.v[i].numpy() for i in range(T) if st.qstep[i]], 1)
    Ut = np.stack([st.u[i].numpy() for i in range(T) if not st.qstep[i]], 1)
    np.testing.assert_allclose(Vq.T @ Vq, np.eye(Vq.shape[1]), atol=1e-13)
    np.testing.assert_allclose(Ut.T @ Ut, np.eye(Ut.shape[1]), atol=1e-13)


def test_step_limits():
    with pytest.raises(ValueError):
        HaarOracle(5, 6, seed=0)
    with pytest.raises(ValueError):
        GinibreOracle(4, 6, 5, seed=0)
    st = HaarOracle(4, 2, seed=0)
    st.apply(np.ones(4))
    st.apply(np.ones(4))
    with pytest.raises(ValueError):
        st.apply(np.ones(4))


def test_zero_input_step():
    """x_t = 0 (e.g. ISTA from x_0 = 0): H_t(0) = I and the output is 0."""
    st = GinibreOracle(6, 6, 3, seed=1)
    y = st.apply(np.zeros(6)).numpy()
    np.testing.assert_array_equal(y, 0.0)
    assert st.R[0].identity
    st2 = HaarOracle(6, 3, seed=1)
    y2 = st2.apply(np.zeros(6)).numpy()
    np.testing.assert_array_equal(y2, 0.0)
