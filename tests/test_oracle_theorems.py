"""Monte-Carlo pins of Theorems 1 and 2: HD and the direct simulation have the same law.

Theorem 1 (Ginibre) and Theorem 2 (Haar) state that the joint law of the trajectory {x_t}
from HD equals the one obtained with a dense Q drawn in advance.  These tests run the
oracle over many trials (the Philox trial word separates them) and the direct simulation
with numpy matrices, and compare the two samples with two-sample Kolmogorov-Smirnov tests
(Bonferroni-corrected over the statistics of one test).  They also check the law of the
fully revealed Q at T = n against textbook facts:
  * Ginibre: the entries of sum_i u_i v_i^T are i.i.d. N(0, 1);
  * Haar: Q_11^2 ~ Beta(1/2, (n-1)/2) (first coordinate of a uniform point on S^{n-1}).
"""
import numpy as np
import pytest
from scipy import stats

from oracle import direct
from oracle.dynamics import f_sign_mem, f_tanh, run
from oracle.hd import GinibreOracle, HaarOracle

ALPHA = 1e-3


def _ks_all(a, b, names):
    k = a.shape[1]
    for j in range(k):
        p = stats.ks_2samp(a[:, j], b[:, j]).pvalue
        assert p > ALPHA / k, f"{names[j]}: KS p={p:.2e}"


def _haar_stats(xs, ys):
    return [ys[0][0], ys[1][0], ys[2][-1], ys[3][3], xs[4][0] * xs[3][1],
            float(np.dot(xs[2], xs[1])) / len(xs[1])]


def test_theorem2_haar_trajectory_law():
    n, T, trials = 40, 4, 1200
    pattern = lambda t: t % 2 == 0
    rng = np.random.default_rng(2024)
    hd, dr = [], []
    for i in range(trials):
        x1 = rng.standard_normal(n)
        xs, ys = run(HaarOracle(n, T, seed=77, trial=i), x1, T, f_sign_mem, pattern)
        hd.append(_haar_stats(xs, ys))
        x1b = rng.standard_normal(n)
        xs, ys = run(direct.DirectState(direct.haar(rng, n)), x1b, T, f_sign_mem, pattern)
        dr.append(_haar_stats(xs, ys))
    names = ["y1[0]", "y2[0]", "y3[-1]", "y4[3]", "x5[0]x4[1]", "x3.x2/n"]
    _ks_all(np.array(hd), np.array(dr), names)


def test_theorem1_ginibre_trajectory_law():
    m, n, T, trials = 24, 32, 5, 1200
    sigma = 1.0 / np.sqrt(m)
    pattern = lambda t: t % 2 == 0
    rng = np.random.default_rng(77)
    def traj(state, x1):
        x, out = x1, []
        for t in range(1, T + 1):
            y = np.asarray(state.apply(x, transpose=pattern(t)), dtype=np.float64)
            out.append(y)
            x = np.tanh(y)
        return out
    hd, dr = [], []
    for i in range(trials):
        ys = traj(GinibreOracle(m, n, T, seed=5, trial=i, sigma=sigma), rng.standard_normal(n))
        hd.append([ys[0][0], ys[1][1], ys[2][-1], ys[3][2], ys[4][0], float(ys[4] @ ys[4]) / n])
        ys = traj(direct.DirectState(direct.ginibre(rng, m, n, sigma)), rng.standard_normal(n))
        dr.append([ys[0][0], ys[1][1], ys[2][-1], ys[3][2], ys[4][0], float(ys[4] @ ys[4]) / n])
    _ks_all(np.array(hd), np.array(dr), ["y1[0]", "y2[1]", "y3[-1]", "y4[2]", "y5[0]", "|y5|^2/n"])


def test_revealed_ginibre_matrix_is_iid_gaussian():
    n, trials = 5, 1500
    rng = np.random.default_rng(3)
    ent = []
    for i in range(trials):
        st = GinibreOracle(n, n, n, seed=19, trial=i)
        run(st, rng.standard_normal(n), n, f_tanh, lambda t: False)
        ent.append(st.revealed().numpy().ravel())
    ent = np.array(ent)
    for j in (0, 7, 12, 24):
        assert stats.kstest(ent[:, j], "norm").pvalue > ALPHA / 4
    c = np.corrcoef(ent.T)
    off = c[~np.eye(n * n, dtype=bool)]
    assert np.max(np.abs(off)) < 0.15


def test_revealed_haar_matrix_first_entry_law():
    n, trials = 6, 1500
    rng = np.random.default_rng(4)
    q11, q66 = [], []
    for i in range(trials):
        st = HaarOracle(n, n, seed=23, trial=i)
        run(st, rng.standard_normal(n), n, f_sign_mem, lambda t: t % 2 == 0)
        Q = st.dense().numpy()
        q11.append(Q[0, 0] ** 2)
        q66.append(Q[-1, -1] ** 2)
    law = stats.beta(0.5, (n - 1) / 2.0)
    assert stats.kstest(q11, law.cdf).pvalue > ALPHA / 2
    assert stats.kstest(q66, law.cdf).pvalue > ALPHA / 2


def test_a_wrong_sign_rule_is_caught():
    """Planted mistake (in a subclass of the oracle's reflector, on the CPU): with
    u = v - s||v||e1 the reflector maps v to -||v||e1.  In Haar's first step the two flips
    cancel, but eq. (Householder_property) and Ginibre's first step Q x_1 = ||x_1|| g_1 both
    catch it."""
    import torch
    from oracle import hd as hdmod
    from oracle import philox

    class Flipped(hdmod.Reflector):
        def __init__(self, k, p):
            super().__init__(k, p)
            if not self.identity:
                a = hdmod._vec(p)[k:]
                e1 = torch.zeros_like(a)
                e1[0] = 1.0
                self.u = a - self.s * self.alpha * e1
                self.uu = torch.dot(self.u, self.u)

    n = 12
    x = np.random.default_rng(1).standard_normal(n)
    Hx = Flipped(0, x).apply(x).numpy()
    assert abs(Hx[0] - np.linalg.norm(x)) > 1.0          # property H v = ||v|| e_1 fails
    g = philox.normals(4, 0, 1, 0, n)
    expect = np.linalg.norm(x) * g
    orig = hdmod.Reflector
    hdmod.Reflector = Flipped
    try:
        y = hdmod.GinibreOracle(n, n, 2, seed=4).apply(x).numpy()
    finally:
        hdmod.Reflector = orig
    assert np.max(np.abs(y - expect)) > 0.1


def test_revealed_haar_matrix_trace_moments():
    """The whole revealed Q at T = n against the trace moments of the Haar measure on O(n)
    (Diaconis and Shahshahani, 1994): for sum_j j a_j <= n/2, E prod_j (tr Q^j)^{a_j} equals
    the same moment of independent sqrt(j) Z_j + [j even].  At n = 8 that fixes
    E tr Q = 0, E (tr Q)^2 = 1, E tr Q^2 = 1, E (tr Q)^4 = 3 and E (tr Q^2)^2 = 3.  The
    trace mixes every diagonal entry, so it sees the joint law, not one entry's marginal.
    A planted mistake (on the CPU, in a subclass of the oracle's reflector) that drops the
    sign factor -s of eq. Householder fails it."""
    import torch
    from oracle import hd as hdmod

    def gaps(trials):
        rng = np.random.default_rng(8)
        t1, t2 = [], []
        for i in range(trials):
            st = hdmod.HaarOracle(8, 8, seed=41, trial=i)
            run(st, rng.standard_normal(8), 8, f_sign_mem, lambda t: t % 3 == 0)
            Q = st.dense().numpy()
            t1.append(np.trace(Q))
            t2.append(np.trace(Q @ Q))
        t1, t2 = np.array(t1), np.array(t2)
        out = []
        for sample, want in ((t1, 0.0), (t1 ** 2, 1.0), (t2, 1.0), (t1 ** 4, 3.0), (t2 ** 2, 3.0)):
            out.append(abs(sample.mean() - want) / (sample.std(ddof=1) / np.sqrt(trials)))
        return np.array(out)

    g = gaps(1000)
    assert (g <= 4.5).all(), g

    class Unsigned(hdmod.Reflector):
        def apply(self, w):
            w = hdmod._vec(w)
            if self.identity:
                return w.clone()
            seg = w[self.k:]
            seg = seg - (2.0 * torch.dot(self.u, seg) / self.uu) * self.u
            return torch.cat([w[:self.k], seg])

    orig = hdmod.Reflector
    hdmod.Reflector = Unsigned
    try:
        bad = gaps(400)
    finally:
        hdmod.Reflector = orig
    assert bad.max() > 4.5, bad
