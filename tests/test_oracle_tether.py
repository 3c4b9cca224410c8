"""Pins of the oracle's tethered / clamped filaments (Sec. 5.2.1, eqs.
tethering_constraint, tethered_rotation_constraint,
tethering_constraint_force_and_torque), independent of its own formulas:

* a clamped filament under a tip force of fixed direction relaxes to the
  elastica of Sec. 4.1 (closed form by quadrature, tests/elastica.py) with the
  L2 error of the tangent angles falling at second order in the segment length,
* at equilibrium the multipliers balance the loads: lambda_1 = -sum F_ext and
  lambda_2 = -sum T_ext - sum (Y_n - Y_1) x F_ext (net force and moment),
* a stiff filament on the motor (prescribed circular base motion and base
  rotation) turns rigidly: its base sits on the circle and its first segment's
  quaternion is exp(j w dt e_z) q_1^0 to rounding, and the free end stays at
  the rigid distance from the axis,
* J0 of a tethered filament is the finite-difference Jacobian of the
  drag-only f_0 at a straight state (where App. B.2's approximations are exact)
  for the clamp, and of the filament-RPY f_0 at a straight unloaded state,
* an all-false mask is the free filament, bit for bit.
"""
import math

import numpy as np
import pytest

import elastica
from oracle import filament as fo
from paper_1903_12609_gb300.inputs import random_frames


def _fd_jacobian(fun, X, h=1e-6):
    f0 = fun(X)
    J = np.empty((f0.size, X.size))
    for k in range(X.size):
        e = np.zeros_like(X)
        e[k] = h
        J[:, k] = (fun(X + e) - fun(X - e)) / (2 * h)
    return J


def _clamp(M, Y1=None):
    return fo.Tether(mask=np.ones(M, dtype=bool),
                     Y1=np.zeros((M, 3)) if Y1 is None else np.asarray(Y1, dtype=np.float64),
                     u1=np.zeros((M, 3)))


def _relax(lay, p, st, ext, teth, max_steps=100):
    """Steps until no position moves by more than the Broyden tolerance."""
    for j in range(max_steps):
        st, _ = fo.step(lay, p, st, ext, tether=teth)
        if j > 3 and np.abs(st.Y - st.Yprev).max() < p.tol * p.a:
            return st
    raise AssertionError("no steady state after %d steps" % max_steps)


def _elastica_error(N, ell=44.0, KB=1.0):
    """Clamped at Y_1 = 0 with tangent e_x, force -F e_z on the last segment,
    F = 1.93 K_B / l^2 with l = (N - 1) dL the arc length from the clamp to
    the loaded segment; returns (E_2, multipliers, steady state)."""
    dL = ell / (N - 1)
    F = 1.93 * KB / ell ** 2
    a = dL / 2.2
    zeta = 6.0 * math.pi * a / dL                  # drag per unit length of the segments
    tau = zeta * ell ** 4 / (12.4 * KB)            # slowest bending relaxation time
    p = fo.Params(a=a, eta=1.0, dL=dL, KB=KB, KT=KB, dt=0.5 * tau, tol=1e-9, max_iter=200)
    lay = fo.Layout([N])
    st = fo.initial_state(lay, p, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]),
                          np.array([[0.0, 1.0, 0.0]]))
    Fext = np.zeros((N, 3))
    Fext[-1] = [0.0, 0.0, -F]
    st = _relax(lay, p, st, fo.External(Fext=Fext), _clamp(1))
    t = fo.frames(st.q)[0]
    th = np.arccos(np.clip(-t[:, 2], -1.0, 1.0))   # angle to the force direction
    th_ex = elastica.angles(dL * np.arange(N), ell, F, KB)
    return math.sqrt(dL * np.sum((th - th_ex) ** 2)), st.tlam[0], st


def test_clamped_elastica_converges_at_second_order():
    E = [_elastica_error(N)[0] for N in (6, 11, 21)]
    # halving dL divides the error by ~4
    assert 3.6 < E[0] / E[1] < 4.8, E
    assert 3.6 < E[1] / E[2] < 4.8, E
    assert E[2] < 4e-4


def test_clamped_multipliers_balance_the_loads():
    """Equilibrium of a clamped filament under gravity plus constant torques,
    the clamp away from the origin."""
    rng = np.random.default_rng(3)
    N = 12
    lay = fo.Layout([N])
    L = N * 2.2
    tau = 6.0 * math.pi / 2.2 * L ** 4 / (12.4 * 400.0)    # slowest bending relaxation
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=400.0, KT=300.0, dt=0.5 * tau, tol=1e-10,
                  max_iter=200)
    base = np.array([[1.5, -2.0, 3.0]])
    t, mu = random_frames(rng, 1)
    st = fo.initial_state(lay, p, base, t, mu)
    Fext = np.tile([0.0, 0.0, -0.02], (N, 1)) + 0.005 * rng.standard_normal((N, 3))
    Text = 0.01 * rng.standard_normal((N, 3))
    st = _relax(lay, p, st, fo.External(Fext=Fext, Text=Text), _clamp(1, base))
    lam1, lam2 = st.tlam[0, :3], st.tlam[0, 3:]
    np.testing.assert_allclose(lam1, -Fext.sum(axis=0), rtol=0, atol=1e-9)
    moment = Text.sum(axis=0) + np.cross(st.Y - st.Y[0], Fext).sum(axis=0)
    np.testing.assert_allclose(lam2, -moment, rtol=0, atol=1e-8)
    np.testing.assert_allclose(st.Y[0], base[0], rtol=0, atol=1e-12)


def test_motor_turns_a_stiff_filament_rigidly():
    """Sec. 5.2.1's set-up at a low Sperm number: base offset delta_0 = 4.5977a
    from the motor axis e_z, filament at 15 degrees to the axis (tilted away
    from it), Y_1 = delta_0 (cos jw dt, sin jw dt, 0), u_1 = (0, 0, w dt)."""
    N, a, dL = 20, 1.0, 2.2
    L = N * dL
    delta0 = 4.5977 * a
    w = 0.02
    zeta = 4.0 * math.pi / (math.log(L / a) + 0.5)
    KB = zeta * w * L ** 4 / 0.1                       # Sp = 0.1
    dt = 2.0 * math.pi / w / 80.0                      # 80 steps per turn
    lay = fo.Layout([N])
    p = fo.Params(a=a, eta=1.0, dL=dL, KB=KB, KT=KB, dt=dt, tol=1e-9, max_iter=100)
    th = math.radians(15.0)
    t0 = np.array([[math.sin(th), 0.0, math.cos(th)]])
    st = fo.initial_state(lay, p, np.array([[delta0, 0.0, 0.0]]), t0, np.array([[0.0, 1.0, 0.0]]))
    q10 = st.q[0].copy()
    u1 = np.array([[0.0, 0.0, w * dt]])
    for j in range(1, 41):                             # half a turn
        ph = j * w * dt
        teth = fo.Tether(mask=np.array([True]),
                         Y1=np.array([[delta0 * math.cos(ph), delta0 * math.sin(ph), 0.0]]), u1=u1)
        st, _ = fo.step(lay, p, st, None, tether=teth)
        np.testing.assert_allclose(st.Y[0], teth.Y1[0], rtol=0, atol=1e-12)
        qz = fo.qexp(np.array([0.0, 0.0, ph]))
        np.testing.assert_allclose(st.q[0], fo.qmul(qz, q10), rtol=0, atol=1e-12)
    d = math.hypot(st.Y[-1, 0], st.Y[-1, 1])
    d_rigid = delta0 + (N - 1) * dL * math.sin(th)
    assert abs(d - d_rigid) < 0.01 * d_rigid, (d, d_rigid)


@pytest.mark.parametrize("bdf2", [False, True])
def test_tethered_J0_equals_fd_jacobian_of_drag_model_when_straight(bdf2):
    rng = np.random.default_rng(7)
    lay = fo.Layout([5, 4])
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=1.5, KT=0.7, dt=0.05, tol=1e-12)
    t, mu = random_frames(rng, 2)
    base = np.array([[0.0, 0.0, 0.0], [20.0, 0.0, 0.0]])
    st = fo.initial_state(lay, p, base, t, mu)
    if bdf2:
        st.Yprev = st.Y + 0.01
        st.u = 0.01 * rng.standard_normal((lay.S, 3))
    teth = fo.Tether(mask=np.array([True, False]), Y1=base, u1=np.zeros((2, 3)))
    Y1 = np.array([rng.standard_normal(3), st.Y[lay.off_seg[1]]])
    u = np.zeros((lay.S, 3))
    u[0] = rng.standard_normal(3)                      # lambda_2 of the tethered filament
    X = lay.join_X(Y1, u, rng.standard_normal((lay.n_lam, 3)))
    J0 = fo.jacobian0_tethered(lay, p, st, X, teth, "drag")

    def f0(Xv):
        return fo.residual(lay, p, st, None, Xv, mob=fo.drag_mobility, tether=teth)

    Jfd = _fd_jacobian(f0, X)
    for i, n in enumerate(lay.N):
        b = lay.off_X[i]
        blk = Jfd[b:b + 6 * n, b:b + 6 * n]
        np.testing.assert_allclose(J0[i], blk, rtol=0, atol=1e-8 * np.abs(blk).max())


def test_tethered_filament_rpy_J0_equals_fd_jacobian_when_straight_and_unloaded():
    rng = np.random.default_rng(8)
    lay = fo.Layout([5])
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=1.5, KT=0.7, dt=0.05, tol=1e-12)
    t, mu = random_frames(rng, 1)
    st = fo.initial_state(lay, p, np.zeros((1, 3)), t, mu)
    teth = _clamp(1)
    X = np.zeros(6 * lay.S)
    J0 = fo.jacobian0_tethered(lay, p, st, X, teth, "rpy")[0]
    Jfd = _fd_jacobian(lambda Xv: fo.residual(lay, p, st, None, Xv, tether=teth), X)
    np.testing.assert_allclose(J0, Jfd, rtol=0, atol=1e-8 * np.abs(Jfd).max())


def test_all_false_mask_is_the_free_filament():
    rng = np.random.default_rng(9)
    lay = fo.Layout([6, 3])
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=1.5, KT=0.7, dt=0.05, tol=1e-12)
    t, mu = random_frames(rng, 2)
    st = fo.initial_state(lay, p, rng.uniform(0, 20, (2, 3)), t, mu)
    X = lay.join_X(np.array([st.Y[0], st.Y[6]]), 0.1 * rng.standard_normal((lay.S, 3)),
                   rng.standard_normal((lay.n_lam, 3)))
    off = fo.Tether(mask=np.zeros(2, dtype=bool), Y1=np.ones((2, 3)), u1=np.ones((2, 3)))
    np.testing.assert_array_equal(fo.residual(lay, p, st, None, X, tether=off),
                                  fo.residual(lay, p, st, None, X))
    for a, b in zip(fo.jacobian0_tethered(lay, p, st, X, off, "rpy"),
                    fo.jacobian0_general(lay, p, st, X, "rpy")):
        np.testing.assert_array_equal(a, b)
