"""Pins of the oracle's optional pre-filters (Sec. 5.3): the 3x3x3 median against
numpy's median over the 27 clamped shifts, and its defining behaviour on
impulses, constants and monotone ramps."""

import numpy as np

import oracle
import phantoms as ph


def _numpy_median3(v):
    p = np.pad(v, 1, mode="edge")
    nz, ny, nx = v.shape
    stack = [p[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
             for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return np.median(np.stack(stack), axis=0)


def test_median_matches_numpy():
    v = ph.random_volume((13, 11, 9), 121, np.float64)
    np.testing.assert_array_equal(oracle.median3(v), _numpy_median3(v))


def test_median_removes_impulses_and_keeps_constants_and_ramps():
    v = np.full((9, 10, 11), 0.3)
    v[4, 5, 5] = 1.0  # isolated impulse
    np.testing.assert_array_equal(oracle.median3(v), np.full(v.shape, 0.3))
    r = ph.ramp_volume((11, 10, 9), (1, 1, 1), (0.01, 0.02, 0.03))
    # a linear ramp's 27 neighbours are symmetric about the centre value away from
    # the clamped border, so the median is the centre there
    np.testing.assert_allclose(oracle.median3(r)[1:-1, 1:-1, 1:-1], r[1:-1, 1:-1, 1:-1], atol=1e-15)
