"""Host-side arithmetic of bench.py that needs no GPU: the whole-trajectory estimate behind
the oracle's CPU baseline and the reference arm."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench   # noqa: E402


def test_whole_samples_give_their_mean():
    secs, a, b, exact = bench.trajectory_seconds(3, [[1.0, 2.0, 3.0], [2.0, 2.0, 2.0]])
    assert exact and a is None and b is None
    assert secs == pytest.approx(6.0)


def test_linear_cost_is_recovered_from_first_products():
    a, b, T = 0.12, 0.004, 100
    samples = [[a + b * t for t in range(1, 11)], [a + b * t for t in range(1, 8)]]
    secs, fa, fb, exact = bench.trajectory_seconds(T, samples)
    assert not exact
    assert fa == pytest.approx(a) and fb == pytest.approx(b)
    assert secs == pytest.approx(T * a + b * T * (T + 1) / 2)
    value, tsecs, how = bench.oracle_throughput(10 ** 6, T, samples)
    assert value == pytest.approx(1e6 * T * T / secs) and tsecs == pytest.approx(secs)
    assert "extrapolated" in how


def test_noisy_decreasing_sample_falls_back_to_a_constant_cost():
    secs, a, b, exact = bench.trajectory_seconds(50, [[0.3, 0.2, 0.1]])
    assert not exact and b == 0.0 and a == pytest.approx(0.2)
    assert secs == pytest.approx(50 * 0.2)


def test_single_product_sample():
    secs, a, b, _ = bench.trajectory_seconds(10, [[0.5], [0.7]])
    assert b == 0.0 and secs == pytest.approx(6.0)
