"""Pins of the steric barrier reference (oracle/steric.py, Sec. 2.6):
magnitude F^S at contact, zero at and beyond the range 2 chi a, a value of
the quartic profile worked by hand, the neighbour exclusion, Newton's third
law, and zero torque of the central pair forces."""
import numpy as np
import pytest

from oracle import steric


def test_contact_range_and_profile():
    a, FS, chi = 1.0, 7.0, 1.1
    e = np.array([0.0, 0.6, 0.8])
    np.testing.assert_allclose(steric.pair_force(2.0 * a * e, a, FS, chi), FS * e, rtol=1e-15)
    assert np.all(steric.pair_force(2.0 * chi * a * e, a, FS, chi) == 0)
    assert np.all(steric.pair_force(3.0 * a * e, a, FS, chi) == 0)
    # r = 2.1 a: ((4.84 - 4.41) / 0.84)^4 * 2.1 / 2
    want = FS * (0.43 / 0.84) ** 4 * 2.1 / 2.0
    np.testing.assert_allclose(steric.pair_force(2.1 * a * e, a, FS, chi), want * e, rtol=1e-12)
    # r -> 0 between distinct segments: zero vector (r_nm / 2a -> 0)
    assert np.all(steric.pair_force(np.zeros(3), a, FS, chi) == 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_neighbours_excluded_third_law_and_torque(seed):
    rng = np.random.default_rng(seed)
    segs = [5, 3, 4]
    Y = rng.uniform(0.0, 4.0, size=(sum(segs), 3))       # many overlaps
    F = steric.barrier_forces(segs, Y, 1.0, 3.0, 1.1)
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12 * np.abs(F).max())
    np.testing.assert_allclose(np.cross(Y, F).sum(axis=0), 0.0, atol=1e-11 * np.abs(F).max())
    # two adjacent segments of one filament at contact feel nothing from each other
    Y2 = np.array([[0.0, 0, 0], [2.0, 0, 0]])
    assert np.all(steric.barrier_forces([2], Y2, 1.0, 3.0, 1.1) == 0)
    # ... but segments two apart on one filament do
    Y3 = np.array([[0.0, 0, 0], [1.0, 5.0, 0], [2.0, 0, 0]])
    F3 = steric.barrier_forces([3], Y3, 1.0, 3.0, 1.1)
    np.testing.assert_allclose(F3[0], [-3.0, 0, 0], rtol=1e-15)
    np.testing.assert_allclose(F3[2], [3.0, 0, 0], rtol=1e-15)
