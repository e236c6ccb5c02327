"""Pins for the oracle's Philox normal generator (oracle/philox.py).

* Bit-exact agreement of the Philox4x32-10 words with cuRAND's host-side
  PHILOX4_32_10 generator (a library implementation, run on the CPU).  cuRAND's host
  generator emits block b of its output from counter (b >> 16, 0, b & 0xffff, 0) with key
  = seed; comparing several 64-bit seeds over 3 * 65536 blocks exercises every word of
  the counter and key in the round function.
* The uniform map lands in (0, 1] with its exact end points.
* The normals are N(0, 1) (Kolmogorov-Smirnov), uncorrelated within a Box-Muller pair,
  and differ between steps, trials and streams.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox


def _load_curand():
    cands = []
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += [os.path.join(d, "libcurand.so"), os.path.join(d, "libcurand.so.10")]
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_words(seed, count):
    lib = _load_curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1234567, 0xFEDCBA9876543210, 0xFFFFFFFFFFFFFFFF])
def test_philox_words_match_curand_host(seed):
    nblocks = 3 * 65536
    ref = _curand_host_words(seed, 4 * nblocks).reshape(nblocks, 4)
    b = np.arange(nblocks, dtype=np.uint64)
    w = philox.philox4x32(b >> np.uint64(16), 0, b & np.uint64(0xFFFF), 0, seed)
    got = np.stack(w, axis=1).astype(np.uint32)
    np.testing.assert_array_equal(got, ref)


def test_uniform_map_end_points():
    assert philox.uniform53(0, 0) == 2.0 ** -53
    assert philox.uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0
    # the 53-bit integer is (hi << 21) | (lo >> 11): the low 11 bits of lo are dropped
    assert philox.uniform53(0, 0x7FF) == 2.0 ** -53
    assert philox.uniform53(0, 0x800) == 2.0 * 2.0 ** -53
    assert philox.uniform53(1, 0) == (2.0 ** 21 + 1) * 2.0 ** -53


def test_normals_are_standard_gaussian():
    z = philox.normals(seed=7, trial=0, step=1, start=0, count=1_000_000)
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1.0) < 5e-3
    ks = stats.kstest(z, "norm")
    assert ks.pvalue > 1e-3
    # the two members of a Box-Muller pair are independent N(0, 1)
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5e-3
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(z ** 4) - 3.0) < 0.05


def test_normals_depend_on_every_counter_word():
    base = philox.normals(3, 0, 1, 0, 64)
    for kw in ({"trial": 1}, {"step": 2}, {"stream": 1}):
        args = dict(seed=3, trial=0, step=1, start=0, count=64, stream=0)
        args.update(kw)
        other = philox.normals(**args)
        assert np.max(np.abs(other - base)) > 0.1
        assert abs(np.corrcoef(other, base)[0, 1]) < 0.5


def test_normals_are_addressed_by_absolute_index():
    full = philox.normals(11, 2, 5, 0, 101)
    for start in (0, 1, 2, 37, 50):
        part = philox.normals(11, 2, 5, start, 101 - start)
        np.testing.assert_array_equal(part, full[start:])


def test_masked_head_is_zero():
    g = philox.gaussian_vector(5, 0, 3, 10, 4, sigma=0.5)
    assert np.all(g[:4] == 0.0)
    np.testing.assert_array_equal(g[4:], 0.5 * philox.normals(5, 0, 3, 4, 6))
