"""Pins of the oracle's interface observables (line crossings) on profiles
whose crossing points are known exactly."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _line(values, ny=3):
    return np.tile(np.asarray(values, dtype=np.float64), (ny, 1))


def test_linear_profile_crossing_is_exact():
    # phi = 0.25 (x - 7.4) is exact under linear interpolation
    x = np.arange(20.0)
    phi = _line(0.25 * (x - 7.4))
    w = np.ones_like(phi)
    fl = _line(np.clip((x - 3.0) / 10.0, 0.0, 1.0))  # s = 1 - fl crosses 1/2 at x = 8
    xp, xs = O.crossings(phi, w, fl, axis=0, index=1)
    assert xp == pytest.approx(7.4, abs=1e-12)
    assert xs == pytest.approx(8.0, abs=1e-12)


def test_last_crossing_along_the_line_and_columns():
    # two crossings of phi along y (rising through 0 at 2.5, falling at 11.75)
    y = np.arange(16.0)
    col = np.where(y < 7, y - 2.5, 11.75 - y)
    phi = np.tile(col[:, None], (1, 4))
    w = np.zeros_like(phi)  # no material: s = -1/2 everywhere, no ice front
    fl = np.ones_like(phi)
    xp, xs = O.crossings(phi, w, fl, axis=1, index=2)
    assert xp == pytest.approx(11.75, abs=1e-12)
    assert math.isnan(xs)


def test_no_crossing_and_node_values_on_the_level():
    phi = _line(np.full(10, 0.3))
    w, fl = np.ones_like(phi), np.zeros_like(phi)  # all ice: s = 1/2 above the level everywhere
    xp, xs = O.crossings(phi, w, fl, axis=0, index=0)
    assert math.isnan(xp) and math.isnan(xs)
    # a node exactly on the level is one crossing, located at that node
    v = np.array([1.0, 0.5, 0.0, -1.0, -2.0])
    xp, _ = O.crossings(_line(v), w[:, :5], fl[:, :5], axis=0, index=2)
    assert xp == 2.0
