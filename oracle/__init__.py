"""Plain, slow CPU FP64 oracle of Householder Dice (arXiv 2101.07464).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import or run anything here.  The CUDA product path never does,
and this package imports nothing from it.

Modules:
  philox    the Philox4x32-10 counter-based normal generator (the oracle's own copy)
  hd        the reflectors of eqs. (Householder)/(Householder_e) and Algorithms 1 and 2,
            one reflector at a time, torch float64 on the CPU
  direct    dense-Q direct simulation for the Monte-Carlo checks of Theorems 1 and 2
  dynamics  the workloads' f_t of eq. (dynamics) in numpy

Every function is pinned by the `-m "not gpu"` tests against facts the paper and the
mathematics fix (closed forms of the first steps, orthogonality, reconstruction of Q at
T = n, distributional equality with the direct simulation, cuRAND's Philox).
"""
