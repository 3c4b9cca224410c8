"""Pins of the oracle's quaternion / Lie-group functions (paper Sec. 2.9, App. A).

* R(q) against the sandwich product q (0,w) q^* that the paper states it equals,
  and against scipy's rotation-vector routine (Rodrigues) through exp(u),
* the square root's properties (a) unit and (b) squares back, App. A.1,
* the single-axis example of Sec. 2.9.3 (Omega = alpha e_z),
* dexpinv through its defining ODE: if du/dt = dexpinv_u(Omega) then
  d/dt exp(u) = (1/2)(0, Omega) exp(u) (finite differences),
* the frame-to-quaternion initialisation of App. A.1.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import filament as fo


def _rand_unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def test_rotation_matrix_is_sandwich_product():
    rng = np.random.default_rng(0)
    q = _rand_unit_quats(rng, 20)
    w = rng.standard_normal((20, 3))
    wq = np.concatenate([np.zeros((20, 1)), w], axis=1)
    sandwich = fo.qmul(fo.qmul(q, wq), fo.qconj(q))
    np.testing.assert_allclose(sandwich[:, 0], 0.0, atol=1e-15)
    np.testing.assert_allclose(sandwich[:, 1:], np.einsum("nij,nj->ni", fo.rotation_matrix(q), w),
                               rtol=1e-13, atol=1e-14)
    R = fo.rotation_matrix(q)
    np.testing.assert_allclose(np.einsum("nki,nkj->nij", R, R), np.broadcast_to(np.eye(3), R.shape),
                               atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)
    p = _rand_unit_quats(rng, 20)
    np.testing.assert_allclose(fo.rotation_matrix(fo.qmul(p, q)),
                               fo.rotation_matrix(p) @ fo.rotation_matrix(q), atol=1e-14)


def test_exp_matches_rotation_vector():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((30, 3)) * rng.uniform(0, 3, size=(30, 1))
    u[0] = 0.0
    u[1] = [1e-9, 0, 0]
    q = fo.qexp(u)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(fo.rotation_matrix(q), Rotation.from_rotvec(u).as_matrix(),
                               atol=1e-14)


def test_single_axis_example():
    """Omega = alpha e_z, q(0) = identity: u = alpha t e_z, q = (cos(at/2),0,0,sin(at/2))."""
    alpha = 0.7
    for t in (0.0, 0.3, 2.0, 5.0):
        u = np.array([0.0, 0.0, alpha * t])
        # u(t) = alpha t e_z solves du/dt = dexpinv_u(Omega): u x Omega = 0
        np.testing.assert_allclose(fo.dexpinv(u, np.array([0, 0, alpha])), [0, 0, alpha],
                                   atol=1e-15)
        np.testing.assert_allclose(fo.qexp(u), [math.cos(alpha * t / 2), 0, 0,
                                                math.sin(alpha * t / 2)], atol=1e-15)


def test_sqrt_properties():
    rng = np.random.default_rng(2)
    p = _rand_unit_quats(rng, 50)
    s = fo.qsqrt(p)
    np.testing.assert_allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(fo.qmul(s, s), p, atol=1e-14)
    np.testing.assert_array_equal(fo.qsqrt(np.array([-1.0, 0, 0, 0])), [0, 0, 0, 1])
    np.testing.assert_allclose(fo.qmul(fo.qsqrt(np.array([-1.0, 0, 0, 0])),
                                       fo.qsqrt(np.array([-1.0, 0, 0, 0]))), [-1, 0, 0, 0])


@pytest.mark.parametrize("scale", [1e-4, 1e-2, 0.3, 1.5, 3.0])
def test_dexpinv_solves_the_quaternion_ode(scale):
    rng = np.random.default_rng(int(scale * 1e4))
    q0 = _rand_unit_quats(rng, 1)[0]
    for _ in range(5):
        u = rng.standard_normal(3)
        u *= scale / np.linalg.norm(u)
        W = rng.standard_normal(3)
        du = fo.dexpinv(u, W)
        h = 1e-6
        qp = fo.qmul(fo.qexp(u + h * du), q0)
        qm = fo.qmul(fo.qexp(u - h * du), q0)
        dq = (qp - qm) / (2 * h)
        rhs = 0.5 * fo.qmul(np.concatenate([[0.0], W]), fo.qmul(fo.qexp(u), q0))
        np.testing.assert_allclose(dq, rhs, rtol=0, atol=1e-8)


def test_dexpinv_series_branch_is_continuous():
    x = np.array([1e-2 * (1 - 1e-9), 1e-2 * (1 + 1e-9)])
    c = fo.dexpinv_coefficient(x)
    assert abs(c[0] - c[1]) < 1e-12
    np.testing.assert_allclose(fo.dexpinv_coefficient(np.array([0.0])), -1 / 12, rtol=1e-15)


def test_quaternion_from_frame():
    rng = np.random.default_rng(3)
    from paper_1903_12609_gb300.inputs import random_frames
    t, mu = random_frames(rng, 40)
    t = np.vstack([t, [[1, 0, 0], [0, 0, 1], [-1, 0, 0], [math.sin(0.7), 0, math.cos(0.7)]]])
    mu = np.vstack([mu, [[0, 1, 0], [0, 1, 0], [0, -1, 0], [0, 1, 0]]])
    q = fo.quat_from_frame(t, mu)
    R = fo.rotation_matrix(q)
    np.testing.assert_allclose(R[:, :, 0], t, atol=1e-14)
    np.testing.assert_allclose(R[:, :, 1], mu, atol=1e-14)
    np.testing.assert_allclose(R[:, :, 2], np.cross(t, mu), atol=1e-14)
