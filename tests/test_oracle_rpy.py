"""Pins of the RPY oracle (paper Sec. 2.7.1) to facts other than itself.

* hand-evaluated closed forms at r = 3a and at contact (tests/golden),
* the self term 1/(6 pi eta a), 1/(8 pi eta a^3),
* continuity of every block across r = 2a and the r -> 0 limit of the
  overlap form (the overlap coefficients are not printed in the paper),
* Faxen-type identities: the rotational blocks equal half the curl of the
  translational / rotlet velocity fields (finite differences),
* the translational block as the double surface average of the Oseen tensor
  (quadrature), for separated and overlapping spheres,
* symmetry and positive-definiteness of the assembled mobility matrix.
"""
import math
import os

import numpy as np
import pytest

from oracle import rpy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rpy_two_sphere.txt")


def _golden():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            r, blk, i, j, num, den = line.split()
            rows.append((float(r), blk, int(i), int(j), float(num) / (float(den) * math.pi)))
    return rows


def test_two_sphere_closed_forms():
    rows = _golden()
    assert len(rows) == 20
    for r in (2.0, 3.0):
        tt, tr, rt, rr = rpy.pair_blocks([r, 0.0, 0.0], False)
        blocks = {"tt": tt, "tr": tr, "rt": rt, "rr": rr}
        expect = {k: np.zeros((3, 3)) for k in blocks}
        for rr_, blk, i, j, val in rows:
            if rr_ == r:
                expect[blk][i, j] = val
        for k in blocks:
            np.testing.assert_allclose(blocks[k], expect[k], rtol=1e-14, atol=1e-16, err_msg=k)


@pytest.mark.parametrize("a,eta", [(1.0, 1.0), (1.5, 0.7)])
def test_self_mobility(a, eta):
    Y = np.array([[0.3, -1.0, 2.0]])
    FT = np.array([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0]])
    VW = rpy.apply(Y, FT, a, eta)
    np.testing.assert_allclose(VW[0, :3], FT[0, :3] / (6 * math.pi * eta * a), rtol=1e-15)
    np.testing.assert_allclose(VW[0, 3:], FT[0, 3:] / (8 * math.pi * eta * a ** 3), rtol=1e-15)


def test_continuity_at_contact():
    rng = np.random.default_rng(1)
    for _ in range(5):
        e = rng.standard_normal(3)
        e /= np.linalg.norm(e)
        a = 1.3
        lo = rpy.pair_blocks(e * 2 * a * (1 - 1e-12), False, a, 0.9)
        hi = rpy.pair_blocks(e * 2 * a * (1 + 1e-12), False, a, 0.9)
        for x, y in zip(lo, hi):
            np.testing.assert_allclose(x, y, rtol=0, atol=1e-10 * np.abs(y).max())


def test_overlap_limit_is_self_term():
    a, eta = 0.8, 1.2
    self_blocks = rpy.pair_blocks([0.0, 0.0, 0.0], True, a, eta)
    for d in ([1e-9, 0, 0], [0, 3e-10, -1e-10], [0.0, 0.0, 0.0]):
        near = rpy.pair_blocks(d, False, a, eta)
        for x, y in zip(near, self_blocks):
            np.testing.assert_allclose(x, y, rtol=0, atol=1e-8 * np.abs(self_blocks[0]).max())
    # two coincident but distinct segments: each sees twice the self mobility
    Y = np.zeros((2, 3))
    FT = np.array([[1.0, 0, 0, 0, 0, 1.0], [1.0, 0, 0, 0, 0, 1.0]])
    VW = rpy.apply(Y, FT, a, eta)
    np.testing.assert_allclose(VW[:, 0], 2 / (6 * math.pi * eta * a), rtol=1e-15)
    np.testing.assert_allclose(VW[:, 5], 2 / (8 * math.pi * eta * a ** 3), rtol=1e-15)


def _curl(field, x, h=1e-5):
    """Central-difference curl of a vector field R^3 -> R^3 at x."""
    J = np.zeros((3, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (field(x + e) - field(x - e)) / (2 * h)
    return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])


@pytest.mark.parametrize("r", [2.0, 2.7, 4.0, 11.0])
def test_rotation_blocks_are_half_curl(r):
    """Faxen's law for rotation: Omega = (1/2) curl u for the far form.

    The translational response to F_m, u(x) = Mtt(x - Y_m) F_m, has curl
    2 Mrt F_m; the rotlet field Mtr(x - Y_m) T_m has curl 2 Mrr T_m."""
    rng = np.random.default_rng(int(r * 10))
    e = rng.standard_normal(3)
    e /= np.linalg.norm(e)
    d0 = e * (r + 1e-3)
    F = rng.standard_normal(3)
    T = rng.standard_normal(3)

    def u_force(d):
        return rpy.pair_blocks(d, False)[0] @ F

    def u_torque(d):
        return rpy.pair_blocks(d, False)[1] @ T

    tt, tr, rt, rr = rpy.pair_blocks(d0, False)
    np.testing.assert_allclose(0.5 * _curl(u_force, d0), rt @ F, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(0.5 * _curl(u_torque, d0), rr @ T, rtol=1e-7, atol=1e-9)


def _fibonacci_sphere(n):
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    phi = math.pi * (1 + 5 ** 0.5) * k
    s = np.sqrt(1 - z ** 2)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _oseen_surface_average(r_vec, a=1.0, n=1500):
    """(1/(4 pi a^2))^2 double surface integral of the Oseen tensor
    G(rho) = (I/rho + rho rho^T/rho^3) / (8 pi) over two spheres of radius a."""
    P = _fibonacci_sphere(n) * a
    acc = np.zeros((3, 3))
    for i in range(0, n, 250):
        rho = r_vec[None, None, :] + P[i:i + 250, None, :] - P[None, :, :]
        rr = np.linalg.norm(rho, axis=-1)
        inv = 1.0 / rr
        acc += np.eye(3) * inv.sum() + np.einsum("abi,abj,ab->ij", rho, rho, inv ** 3)
    return acc / (8 * math.pi) / n ** 2


@pytest.mark.parametrize("r,tol", [(3.0, 2e-4), (1.2, 5e-3), (0.5, 5e-3)])
def test_translation_block_is_surface_averaged_oseen(r, tol):
    """Mtt(r) is the double surface average of the Oseen tensor, for separated
    and for overlapping spheres alike (the identity behind both branches)."""
    r_vec = np.array([0.3, -0.5, 0.81])
    r_vec = r_vec / np.linalg.norm(r_vec) * r
    tt = rpy.pair_blocks(r_vec, False)[0]
    quad = _oseen_surface_average(r_vec)
    scale = 1 / (6 * math.pi)
    np.testing.assert_allclose(quad, tt, rtol=0, atol=tol * scale)


def _dense_matrix(Y, a=1.0, eta=1.0):
    S = Y.shape[0]
    Mx = np.zeros((6 * S, 6 * S))
    for k in range(6 * S):
        e = np.zeros(6 * S)
        e[k] = 1.0
        Mx[:, k] = rpy.apply(Y, e.reshape(S, 6), a, eta).ravel()
    return Mx


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_symmetric_positive_definite(seed):
    rng = np.random.default_rng(seed)
    S = 30
    steps = rng.standard_normal((S, 3))
    steps *= 1.4 / np.linalg.norm(steps, axis=1, keepdims=True)   # overlapping walk
    Y = np.cumsum(steps, axis=0) + rng.uniform(0, 3, size=(S, 3))
    d = np.linalg.norm(Y[:, None] - Y[None], axis=-1)
    assert np.sum((d < 2.0) & (d > 0)) > S          # many overlapping pairs
    Mx = _dense_matrix(Y, 1.0, 1.0)
    np.testing.assert_allclose(Mx, Mx.T, rtol=0, atol=1e-15)
    w = np.linalg.eigvalsh(0.5 * (Mx + Mx.T))
    assert w.min() > 0
    np.linalg.cholesky(Mx)


def test_rows_match_full_apply():
    rng = np.random.default_rng(5)
    Y = rng.uniform(0, 8, size=(50, 3))
    FT = rng.standard_normal((50, 6))
    full, fabs = rpy.apply(Y, FT, with_abs=True)
    rows = np.array([0, 7, 49, 7])
    part, pabs = rpy.apply_rows(Y, FT, rows, with_abs=True)
    np.testing.assert_array_equal(part, full[rows])
    np.testing.assert_array_equal(pabs, fabs[rows])
    assert np.all(fabs >= np.abs(full))


def test_threads_do_not_change_results():
    rng = np.random.default_rng(6)
    Y = rng.uniform(0, 10, size=(200, 3))
    FT = rng.standard_normal((200, 6))
    np.testing.assert_array_equal(rpy.apply(Y, FT, nthreads=1), rpy.apply(Y, FT, nthreads=4))
