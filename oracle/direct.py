"""Direct simulation with a dense Q (test infrastructure only).

The paper's baseline: draw the whole matrix first, then iterate eq. (dynamics)
(Section 1, "direct approach"; Theorems 1 and 2 compare HD against it).  Used only at
small n for the Monte-Carlo checks of Theorems 1 and 2.

  * Gin(m, n): i.i.d. N(0, sigma^2) entries (Section 3 notation).
  * Haar(n): Q R decomposition of a Gaussian matrix with the signs of diag(R) folded
    into Q (Mezzadri 2007, cited in Section 1), which is Haar distributed.
Randomness comes from numpy's PCG64, independent of the Philox draws of the HD oracle.
"""
import numpy as np


def ginibre(rng, m, n, sigma=1.0):
    return sigma * rng.standard_normal((m, n))


def haar(rng, n):
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


class DirectState:
    """Same calling convention as the HD oracles: apply(x, transpose) -> M_t x."""

    def __init__(self, Q):
        self.Q = np.asarray(Q, dtype=np.float64)
        self.t = 0

    def apply(self, x, transpose=False):
        self.t += 1
        x = np.asarray(x, dtype=np.float64)
        return self.Q.T @ x if transpose else self.Q @ x
