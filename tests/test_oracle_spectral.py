"""The spectral method on Householder Dice (Section 2.2), pinned against a dense
computation: at m = 10 the Haar state is fully determined after m products, so D built from
the revealed Q = L_1..L_m R_m..R_1 must reproduce the measurements and every power iterate
the Householder Dice run produced (to rounding)."""
import numpy as np
import torch

import synth
from oracle.hd import HaarOracle
from oracle.spectral import power_iteration


def test_spectral_power_iteration_matches_dense_D():
    n, m, K = 6, 10, 4                      # 1 + 2K = 9 products, one more reveals all of Q
    xi = synth.x1(n, 3)
    x0 = synth.x1(n, 4)
    ora = HaarOracle(m, m, 5)
    y, xs = power_iteration(ora, xi, n, m, K, x0)
    ora.apply(torch.zeros(m, dtype=torch.float64) + 1.0, False)   # the m-th product
    Q = ora.dense().numpy()
    A = Q[:n, :]                             # [I_n 0] Q
    y_dense = np.tanh(np.abs(A.T @ xi))
    np.testing.assert_allclose(y.numpy(), y_dense, rtol=0, atol=1e-13)
    D = A @ np.diag(y_dense) @ A.T / m
    x = x0 / np.linalg.norm(x0)
    for k in range(K):
        v = D @ x
        x = v / np.linalg.norm(v)
        np.testing.assert_allclose(xs[k].numpy(), x, rtol=0, atol=1e-12)


def test_spectral_power_iteration_converges_to_top_eigenvector():
    n, m, K = 6, 200, 60                     # T = 1 + 2K = 121 products <= m
    xi = synth.x1(n, 7)
    ora = HaarOracle(m, 1 + 2 * K, 8)
    y, xs = power_iteration(ora, xi, n, m, K, synth.x1(n, 9))
    # consecutive iterates settle (power iteration on a symmetric PSD matrix)
    assert abs(abs(float(torch.dot(xs[-1], xs[-2]))) - 1.0) <= 1e-6
