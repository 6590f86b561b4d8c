"""Seeded generators: deterministic, and shaped like the stated workloads."""
import math

import numpy as np

from paper_2603_17166_gb300 import synthetic as S


def test_deterministic_and_reality():
    a = S.gaussian_alm(32, 2, S.rng(2, "alm"), "inv_l2")
    b = S.gaussian_alm(32, 2, S.rng(2, "alm"), "inv_l2")
    assert np.array_equal(a, b)
    assert np.all(a[:33].imag == 0)          # m = 0 real
    assert np.all(a[:2] == 0)                # l < 2 (spin 2) zero


def test_cap_and_fields():
    th, ph = S.cap_points(20000, 10.0, S.rng(1, "points"), "S")
    assert np.degrees((math.pi - th).max()) <= 10.0 + 1e-12
    # uniform in area: the median colatitude from the pole is at the half-area radius
    half = math.degrees(math.acos(0.5 * (1 + math.cos(math.radians(10)))))
    assert abs(np.degrees(np.median(math.pi - th)) - half) < 0.1
    th, ph = S.field_points("grid4", "R", S.rng(2, "points"), S.rng(2, "deflections"), step_arcmin=4.0)
    assert 34.0 < np.degrees(th.max()) < 35.5        # smallest enclosing cap of the ~4% field
    th, ph = S.field_points("random1", "S", S.rng(3, "points"), n=5000)
    assert 38.0 < np.degrees((math.pi - th).max()) < 38.76
