"""Reading A15 as a test (no implementation on trial but the oracle): how much the later
outputs of a teacher-forced trajectory move when x_1 changes by one rounding (relative
1e-16), for Haar x_{t+1} = tanh(y_t).

* All Q: the change stays at the rounding level through T = 64.
* Q and Q^T alternating: it grows by orders of magnitude within 64 steps.  This is why
  per-step parity between two correct FP64 implementations is only pinned at 1e-12 where
  the schedule is well conditioned or the trajectory short.
"""
import numpy as np

import synth
from gpu_util import next_input
from oracle.hd import make_oracle


def drift(n, T, sched, seed=41):
    a, b = make_oracle("haar", n, n, T, seed), make_oracle("haar", n, n, T, seed)
    rng = np.random.default_rng(0)
    x = synth.x1(n, seed)
    out = []
    for t in range(1, T + 1):
        ya = a.apply(x, sched(t)).numpy()
        xb = x * (1.0 + 1e-16 * rng.standard_normal(n)) if t == 1 else x
        yb = b.apply(xb, sched(t)).numpy()
        out.append(np.linalg.norm(ya - yb) / np.linalg.norm(ya))
        x = next_input(ya, t + 1, sched(t + 1), n, n, seed)
    return np.array(out)


def test_alternating_schedule_amplifies_rounding_all_q_does_not():
    n, T = 300, 64
    allq = drift(n, T, lambda t: False)
    alt = drift(n, T, lambda t: t % 2 == 0)
    assert allq.max() <= 1e-14, allq.max()
    assert alt[:16].max() <= 1e-14, alt[:16].max()
    assert alt[-1] >= 1e-11, alt[-1]          # grown by more than three orders of magnitude
