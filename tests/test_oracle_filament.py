"""Pins of the oracle's filament model and solver (paper Sec. 2.4-2.9, 3, App. B).

* moments: straight untwisted filament -> 0; a helix (constant relative
  rotation) -> closed form derived from the quaternion algebra; a small planar
  bend -> the planar formula K_B t_n x t_{n+1} / dL of Sec. 2.8.1,
* telescoping invariants of the discrete balances (net constraint force and
  net elastic torque vanish; internal loads exert no net moment when the
  constraint holds),
* residual at rest is exactly zero and the state stays at rest,
* a sedimenting sphere and a sphere pair follow the Stokes / RPY velocities,
* J0 of App. B.2 equals the finite-difference Jacobian of the drag-only f_0
  at a straight, untwisted state (where its approximations are exact),
* Algorithm 2's limited-memory iterates equal the textbook dense bad-Broyden
  update, and a linear problem with J0 = J converges in one iteration,
* a converged timestep equals a finite-difference Newton solve,
* quaternions stay unit across steps (multiplicative update, Sec. 2.9.3),
* BDF2 converges at second order in time on the settling-square problem of
  Sec. 4.2 (scaled down), measured against a run with a 32 times smaller step.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import filament as fo


def _params(**kw):
    base = dict(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.3, dt=0.05, tol=1e-12, max_iter=60)
    base.update(kw)
    return fo.Params(**base)


def _rand_quat(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


def test_straight_untwisted_has_no_moment():
    rng = np.random.default_rng(0)
    p = _params()
    q = np.tile(_rand_quat(rng), (5, 1))
    M = fo.internal_moments(q[:-1], q[1:], p)
    np.testing.assert_allclose(M, 0.0, atol=1e-15)


@pytest.mark.parametrize("theta", [1e-3, 0.4, 1.7])
def test_helix_closed_form(theta):
    """q_{n+1} = r q_n with r a rotation by theta about v: the moment is
    R(q_{n+1/2}) D ((4/dL) sin(theta/4) R(q_n)^T v - (g0, kmu, knu)), with
    q_{n+1/2} the rotation by theta/2 about v applied after q_n."""
    rng = np.random.default_rng(int(theta * 1000))
    p = _params(KB=1.7, KT=0.9, gamma0=0.2, kappa_mu=-0.3, kappa_nu=0.15)
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    r = np.concatenate([[math.cos(theta / 2)], math.sin(theta / 2) * v])
    qn = _rand_quat(rng)
    qn1 = fo.qmul(r, qn)
    M = fo.internal_moments(qn[None], qn1[None], p)[0]
    Rn = Rotation.from_quat(np.roll(qn, -1)).as_matrix()        # scipy is scalar-last
    Rh = Rotation.from_rotvec(theta / 2 * v).as_matrix() @ Rn
    D = np.diag([p.KT, p.KB, p.KB])
    expect = Rh @ D @ ((4 / p.dL) * math.sin(theta / 4) * Rn.T @ v
                       - np.array([p.gamma0, p.kappa_mu, p.kappa_nu]))
    np.testing.assert_allclose(M, expect, rtol=1e-12, atol=1e-13)


def test_small_planar_bend_matches_planar_formula():
    """Bending in the plane normal to nu by a small angle: the 3D moment tends
    to K_B t_n x t_{n+1} / dL (eq. discrete2Dmoments) with O(theta^3) error."""
    p = _params(KB=1.0, KT=5.0)
    for th in (1e-2, 1e-3):
        q0 = fo.quat_from_frame([1.0, 0, 0], [0, 1.0, 0])[0]
        r = np.array([math.cos(th / 2), 0, 0, math.sin(th / 2)])     # about e_z = nu
        q1 = fo.qmul(r, q0)
        M = fo.internal_moments(q0[None], q1[None], p)[0]
        t0 = fo.frames(q0)[0]
        t1 = fo.frames(q1)[0]
        planar = p.KB * np.cross(t0, t1) / p.dL
        assert np.linalg.norm(M - planar) <= th ** 3 * p.KB / p.dL


def _random_filament_state(rng, lay, p, twist=0.3):
    base = rng.standard_normal((lay.M, 3))
    from paper_1903_12609_gb300.inputs import random_frames
    t, mu = random_frames(rng, lay.M)
    xi = twist * rng.standard_normal((lay.S, 3))
    return fo.initial_state(lay, p, base, t, mu, xi)


def test_telescoping_and_net_moment():
    rng = np.random.default_rng(3)
    lay = fo.Layout([7, 4])
    p = _params()
    st = _random_filament_state(rng, lay, p)
    u = 0.2 * rng.standard_normal((lay.S, 3))
    lam = rng.standard_normal((lay.n_lam, 3))
    X = lay.join_X(np.array([st.Y[0], st.Y[7]]), u, lam)
    q, t, Y, _, lam2 = fo.unpack(lay, p, X, st.q)
    F, T = fo.forces_torques(lay, p, q, t, lam2, None)
    for i in range(lay.M):
        s, e = lay.off_seg[i], lay.off_seg[i + 1]
        np.testing.assert_allclose(F[s:e].sum(axis=0), 0.0, atol=1e-13)
        net = T[s:e].sum(axis=0) + np.cross(Y[s:e], F[s:e]).sum(axis=0)
        np.testing.assert_allclose(net, 0.0, atol=1e-12)
    # elastic torques alone also telescope
    F0, T0 = fo.forces_torques(lay, p, q, t, np.zeros_like(lam2), None)
    np.testing.assert_allclose(F0, 0.0, atol=0)
    for i in range(lay.M):
        s, e = lay.off_seg[i], lay.off_seg[i + 1]
        np.testing.assert_allclose(T0[s:e].sum(axis=0), 0.0, atol=1e-13)


def test_rest_state_is_a_solution():
    rng = np.random.default_rng(4)
    lay = fo.Layout([6])
    p = _params()
    from paper_1903_12609_gb300.inputs import random_frames
    t, mu = random_frames(rng, 1)
    st = fo.initial_state(lay, p, np.array([[1.0, 2.0, 3.0]]), t, mu)
    st.Yprev = st.Y.copy()
    st.u = np.zeros((lay.S, 3))
    X0 = fo.initial_guess(lay, st)
    f = fo.residual(lay, p, st, None, X0)
    np.testing.assert_allclose(f, 0.0, atol=1e-14)
    st2, iters = fo.step(lay, p, st, None)
    assert iters == 0
    np.testing.assert_allclose(st2.Y, st.Y, atol=1e-14)
    np.testing.assert_allclose(st2.q, st.q, atol=1e-15)


def test_single_sphere_sediments_at_stokes_velocity():
    lay = fo.Layout([1])
    p = _params(dt=0.3)
    st = fo.State(Y=np.array([[0.0, 0.0, 5.0]]), q=np.array([[1.0, 0, 0, 0]]))
    ext = fo.External(Fext=np.array([[0.0, 0.0, -2.0]]))
    V = -2.0 / (6 * math.pi)
    for j in range(4):
        st, iters = fo.step(lay, p, st, ext)
        # f is linear with J0 = I: one iteration on the first step; afterwards the
        # linear extrapolation of Y_1 is already exact for uniform motion
        assert iters == (1 if j == 0 else 0)
        np.testing.assert_allclose(st.Y[0], [0, 0, 5.0 + (j + 1) * p.dt * V], atol=1e-13)
        np.testing.assert_allclose(st.q[0], [1, 0, 0, 0], atol=1e-15)


def test_sphere_pair_sediments_at_rpy_velocity():
    lay = fo.Layout([1, 1])
    d = 5.0
    p = _params(dt=0.2)
    st = fo.State(Y=np.array([[0.0, 0, 0], [d, 0, 0]]), q=np.tile([1.0, 0, 0, 0], (2, 1)))
    ext = fo.External(Fext=np.array([[0, 0, -1.0], [0, 0, -1.0]]))
    V = -(1 / (6 * math.pi) + (1 + 2 / (3 * d * d)) / (8 * math.pi * d))
    for j in range(3):
        st, _ = fo.step(lay, p, st, ext)
        np.testing.assert_allclose(st.Y[:, 2], (j + 1) * p.dt * V, atol=1e-11)
        np.testing.assert_allclose(st.Y[:, 0], [0, d], atol=1e-11)


def _fd_jacobian(fun, X, h=1e-6):
    f0 = fun(X)
    J = np.zeros((f0.size, X.size))
    for k in range(X.size):
        e = np.zeros_like(X)
        e[k] = h
        J[:, k] = (fun(X + e) - fun(X - e)) / (2 * h)
    return J


@pytest.mark.parametrize("bdf2", [False, True])
def test_J0_equals_fd_jacobian_of_drag_model_when_straight(bdf2):
    rng = np.random.default_rng(5)
    lay = fo.Layout([5])
    p = _params(KB=1.5, KT=0.7)
    from paper_1903_12609_gb300.inputs import random_frames
    t, mu = random_frames(rng, 1)
    st = fo.initial_state(lay, p, np.zeros((1, 3)), t, mu)
    if bdf2:
        st.Yprev = st.Y + 0.01
        st.u = 0.01 * rng.standard_normal((lay.S, 3))
    lam = rng.standard_normal((lay.n_lam, 3))
    X = lay.join_X(st.Y[:1], np.zeros((lay.S, 3)), lam)
    J0 = fo.jacobian0(lay, p, st, X)[0]

    def f0(Xv):
        return fo.residual(lay, p, st, None, Xv, mob=fo.drag_mobility)

    Jfd = _fd_jacobian(f0, X)
    np.testing.assert_allclose(J0, Jfd, rtol=0, atol=1e-8 * np.abs(Jfd).max())


def test_J0_is_close_to_fd_jacobian_when_bent():
    """Away from the straight state J0 is an approximation (Taylor-truncated
    dexpinv, frame-vector moments); it stays a few per cent from the exact
    drag-model Jacobian for a gently bent, twisted filament."""
    rng = np.random.default_rng(6)
    lay = fo.Layout([6])
    p = _params(KB=1.5, KT=0.7)
    st = _random_filament_state(rng, lay, p, twist=0.05)
    lam = 0.3 * rng.standard_normal((lay.n_lam, 3))
    u = 0.05 * rng.standard_normal((lay.S, 3))
    X = lay.join_X(st.Y[:1], u, lam)
    J0 = fo.jacobian0(lay, p, st, X)[0]
    Jfd = _fd_jacobian(lambda Xv: fo.residual(lay, p, st, None, Xv, mob=fo.drag_mobility), X)
    rel = np.linalg.norm(J0 - Jfd) / np.linalg.norm(Jfd)
    assert rel < 0.05


def _dense_bad_broyden(fun, J0inv, X0, iters):
    X = X0.copy()
    f = fun(X)
    H = J0inv.copy()
    out = []
    for _ in range(iters):
        dX = -H @ f
        Xn = X + dX
        fn = fun(Xn)
        df = fn - f
        H = H + np.outer(dX - H @ df, df) / (df @ df)
        X, f = Xn, fn
        out.append(X.copy())
    return out


def test_limited_memory_broyden_equals_dense_update():
    rng = np.random.default_rng(7)
    n = 12
    A = np.eye(n) * 3 + 0.3 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)

    def fun(X):
        return A @ X + 0.2 * np.sin(X) + 0.05 * X ** 3 - b

    J0inv = np.linalg.inv(A)
    X0 = np.zeros(n)
    br = fo.Broyden(fun, lambda v: J0inv @ v, X0, 1e-14)
    dense = _dense_bad_broyden(fun, J0inv, X0, 8)
    for k in range(8):
        X, _ = br.iterate()
        np.testing.assert_allclose(X, dense[k], rtol=1e-12, atol=1e-13)


def test_linear_problem_with_exact_J0_converges_in_one_iteration():
    rng = np.random.default_rng(8)
    n = 9
    A = np.eye(n) + 0.4 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    Ainv = np.linalg.inv(A)
    br = fo.Broyden(lambda X: A @ X - b, lambda v: Ainv @ v, np.zeros(n), 1e-12)
    br.iterate()
    assert br.converged()
    np.testing.assert_allclose(br.X, np.linalg.solve(A, b), rtol=1e-12)


def test_converged_step_equals_newton_solution():
    rng = np.random.default_rng(9)
    lay = fo.Layout([4])
    p = _params(KB=3.0, KT=3.0, dt=0.1, tol=1e-13)
    _, t, mu, xi = (np.zeros((1, 3)), np.array([[0.6, 0, 0.8]]), np.array([[0, 1.0, 0]]),
                    0.05 * rng.standard_normal((4, 3)))
    st = fo.initial_state(lay, p, np.zeros((1, 3)), t, mu, xi)
    ext = fo.External(Fext=np.tile([0, 0, -0.5], (4, 1)))
    br = fo.begin_step(lay, p, st, ext)
    while not br.converged():
        br.iterate()

    def fun(X):
        return fo.residual(lay, p, st, ext, X)

    X = fo.initial_guess(lay, st)
    for _ in range(20):
        f = fun(X)
        if np.abs(f).max() < 1e-14:
            break
        X = X - np.linalg.solve(_fd_jacobian(fun, X, 1e-7), f)
    np.testing.assert_allclose(br.X, X, rtol=0, atol=1e-10)


def test_quaternions_stay_unit_over_steps():
    rng = np.random.default_rng(10)
    lay = fo.Layout([6, 5])
    p = _params(KB=2.0, KT=2.0, dt=0.2, tol=1e-10)
    st = _random_filament_state(rng, lay, p, twist=0.1)
    ext = fo.External(Fext=np.tile([0, 0, -1.0], (lay.S, 1)), follower=np.array([0.0, 0.3]))
    for _ in range(4):
        st, _ = fo.step(lay, p, st, ext)
        np.testing.assert_allclose(np.linalg.norm(st.q, axis=1), 1.0, atol=2e-15)
        # the constraint holds at every committed state
        t = fo.frames(st.q)[0]
        for i in range(lay.M):
            s, e = lay.off_seg[i], lay.off_seg[i + 1]
            g = st.Y[s + 1:e] - st.Y[s:e - 1] - 0.5 * p.dL * (t[s:e - 1] + t[s + 1:e])
            np.testing.assert_allclose(g, 0.0, atol=1e-13)


@pytest.mark.parametrize("history", [False, True])
def test_general_J0_with_drag_mobility_is_the_printed_J0(history):
    """The J0 built from a per-filament mobility matrix reduces to App. B.2's
    printed blocks when that matrix is the diagonal self mobility."""
    rng = np.random.default_rng(11)
    lay = fo.Layout([6, 1, 3])
    p = _params(KB=1.5, KT=0.7, gamma0=0.1, kappa_mu=0.2, kappa_nu=-0.1)
    st = _random_filament_state(rng, lay, p, twist=0.2)
    if history:
        st.Yprev = st.Y + 0.01
        st.u = 0.01 * rng.standard_normal((lay.S, 3))
    Y1 = np.array([st.Y[lay.off_seg[i]] for i in range(lay.M)])
    X = lay.join_X(Y1, 0.1 * rng.standard_normal((lay.S, 3)), rng.standard_normal((lay.n_lam, 3)))
    for a, b in zip(fo.jacobian0(lay, p, st, X), fo.jacobian0_general(lay, p, st, X, "drag")):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())


def test_filament_rpy_J0_equals_fd_jacobian_when_straight_and_unloaded():
    """With the filament's own RPY blocks in f_0, J0 is the exact Jacobian of
    that f_0 at a straight, untwisted, tension-free state (u = 0, Lambda = 0):
    there the derivative approximations are exact and dM/dY multiplies zero
    internal load."""
    rng = np.random.default_rng(12)
    lay = fo.Layout([5])
    p = _params(KB=1.5, KT=0.7)
    from paper_1903_12609_gb300.inputs import random_frames
    t, mu = random_frames(rng, 1)
    st = fo.initial_state(lay, p, np.zeros((1, 3)), t, mu)
    X = lay.join_X(st.Y[:1], np.zeros((lay.S, 3)), np.zeros((lay.n_lam, 3)))
    J0 = fo.jacobian0_general(lay, p, st, X, "rpy")[0]
    Jfd = _fd_jacobian(lambda Xv: fo.residual(lay, p, st, None, Xv), X)
    np.testing.assert_allclose(J0, Jfd, rtol=0, atol=1e-8 * np.abs(Jfd).max())


def test_filament_rpy_J0_cuts_broyden_iterations():
    """Several straight sedimenting filaments: the filament-RPY J0 converges in
    fewer Broyden iterations than the drag-only J0 and to the same solution."""
    from paper_1903_12609_gb300.inputs import cloud_frames, workload_params
    wl = workload_params(6, 16, B=1000.0, dt_over_T=0.005, tol=1e-10)
    base, t, mu, _ = cloud_frames(6, 16, volume_fraction=0.02, seed=3)
    lay = fo.Layout([16] * 6)
    p = fo.Params(a=1, eta=1, dL=2.2, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol, max_iter=200)
    st = fo.initial_state(lay, p, base, t, mu)
    ext = fo.External(Fext=np.tile([0, 0, -2.2], (lay.S, 1)))
    s_drag, it_drag = fo.step(lay, p, st, ext, j0_model="drag")
    s_rpy, it_rpy = fo.step(lay, p, st, ext, j0_model="rpy")
    assert it_rpy < it_drag
    np.testing.assert_allclose(s_rpy.Y, s_drag.Y, rtol=0, atol=1e-8)


def _settling_square(N, n_steps, tf_over_T, tol=1e-12):
    """Sec. 4.2's 3D test, scaled down: four straight vertical filaments at the
    corners of a horizontal square of side 0.268 L (as in Sec. 5.4.3), B = 1000,
    settling for tf under gravity; returns the final positions."""
    from paper_1903_12609_gb300.inputs import workload_params
    wl = workload_params(4, N, B=1000.0, dt_over_T=tf_over_T / n_steps, tol=tol)
    D = 0.268 * wl.extra["L"]
    base = np.array([[0, 0, 0], [D, 0, 0], [0, D, 0], [D, D, 0]], dtype=float)
    lay = fo.Layout([N] * 4)
    p = fo.Params(a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                  max_iter=100)
    st = fo.initial_state(lay, p, base, np.tile([0.0, 0.0, 1.0], (4, 1)),
                          np.tile([1.0, 0.0, 0.0], (4, 1)))
    ext = fo.External(Fext=np.tile([0.0, 0.0, -wl.W * wl.dL], (lay.S, 1)))
    for _ in range(n_steps):
        st, _ = fo.step(lay, p, st, ext)
    return st.Y


@pytest.mark.slow
def test_bdf2_converges_at_second_order_in_time():
    """Maximum position error at t = T/2 for dt = T/20, T/40, T/80 against
    dt = T/640: halving dt divides it by ~4 (the backward-Euler first step
    contributes one O(dt^2) local error only)."""
    ref = _settling_square(8, 320, 0.5)
    err = [np.linalg.norm(_settling_square(8, n, 0.5) - ref, axis=1).max() for n in (10, 20, 40)]
    assert 3.6 < err[0] / err[1] < 4.4, err
    assert 3.6 < err[1] / err[2] < 4.4, err


# --------------------------------------------------------------------------
# Initial guess (Sec. 3.3: guesses extrapolated from past steps; the order is
# a reading, linear by default, quadratic as an option)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", [0, 1, 2])
def test_extrapolation_is_exact_on_polynomials_of_its_degree(order):
    """Samples p(0), p(-1), p(-2), p(-3) of a polynomial of degree order are
    continued exactly to p(1); one degree higher, the error is the leading
    finite difference: for p = c t^(order+1), p(1) - x_0 = (order+1)! c (the
    (order+1)-th backward difference of t^(order+1) at unit spacing)."""
    rng = np.random.default_rng(30)
    coef = rng.standard_normal((order + 2, 4))           # a vector of 4 unknowns

    def p(t, deg):
        return sum(coef[k] * t ** k for k in range(deg + 1))

    hist = [p(-float(j), order) for j in range(4)]
    np.testing.assert_allclose(fo.extrapolate(hist, order), p(1.0, order), rtol=0, atol=1e-13)
    hist = [coef[order + 1] * (-float(j)) ** (order + 1) for j in range(4)]
    err = coef[order + 1] * 1.0 - fo.extrapolate(hist, order)
    np.testing.assert_allclose(err, math.factorial(order + 1) * coef[order + 1], rtol=1e-13)


def test_extrapolation_error_falls_at_the_order_plus_one():
    """On a smooth signal the extrapolation error falls as h^(order+1)."""
    for order in (1, 2):
        errs = []
        for h in (0.02, 0.01):
            hist = [np.array([math.sin(1.0 - j * h)]) for j in range(3)]
            errs.append(abs(fo.extrapolate(hist, order)[0] - math.sin(1.0 + h)))
        assert abs(math.log2(errs[0] / errs[1]) - (order + 1)) < 0.1, (order, errs)


def test_extrapolation_drops_to_the_values_that_exist():
    x = [np.array([3.0]), np.array([1.0]), None, np.array([100.0])]
    np.testing.assert_allclose(fo.extrapolate(x, 2), [5.0])           # linear: 2*3 - 1
    np.testing.assert_allclose(fo.extrapolate(x[:1], 2), [3.0])
    np.testing.assert_allclose(fo.extrapolate(x, 0), [3.0])


def test_quadratic_initial_guess_wires_each_history_level():
    """A state whose Y, u and Lambda histories are quadratic in the step index:
    the order-2 guess is their value at the next step in every slot; with u^{j-2}
    and Lambda^{j-2} missing those fall back to the linear guess while Y_1 stays
    quadratic; order 1 is the linear guess."""
    rng = np.random.default_rng(31)
    lay = fo.Layout([5, 3])
    c = [rng.standard_normal((lay.S, 3)) for _ in range(3)]
    d = [rng.standard_normal((lay.S, 3)) for _ in range(3)]
    e = [rng.standard_normal((lay.n_lam, 3)) for _ in range(3)]

    def quad(k, t):
        return k[0] + k[1] * t + k[2] * t * t

    st = fo.State(Y=quad(c, 0.0), q=np.tile([1.0, 0, 0, 0], (lay.S, 1)), Yprev=quad(c, -1.0),
                  Yprev2=quad(c, -2.0), u=quad(d, 0.0), u_prev=quad(d, -1.0),
                  u_prev2=quad(d, -2.0), lam=quad(e, 0.0), lam_prev=quad(e, -1.0),
                  lam_prev2=quad(e, -2.0), steps=3)
    first = [lay.off_seg[i] for i in range(lay.M)]
    want = lay.join_X(quad(c, 1.0)[first], quad(d, 1.0), quad(e, 1.0))
    np.testing.assert_allclose(fo.initial_guess(lay, st, order=2), want, rtol=0, atol=1e-13)
    lin = lay.join_X(2 * quad(c, 0.0)[first] - quad(c, -1.0)[first],
                     2 * quad(d, 0.0) - quad(d, -1.0), 2 * quad(e, 0.0) - quad(e, -1.0))
    np.testing.assert_allclose(fo.initial_guess(lay, st, order=1), lin, rtol=0, atol=1e-13)
    st.u_prev2 = st.lam_prev2 = None
    mixed = lay.join_X(quad(c, 1.0)[first], 2 * quad(d, 0.0) - quad(d, -1.0),
                       2 * quad(e, 0.0) - quad(e, -1.0))
    np.testing.assert_allclose(fo.initial_guess(lay, st, order=2), mixed, rtol=0, atol=1e-13)


def test_commit_fills_the_history_levels_in_turn():
    """After k committed steps from a fresh state: Y^{j-2} from the second
    commit on, u^{j-1}, Lambda^{j-1} from the second, u^{j-2}, Lambda^{j-2}
    from the third, each equal to the value committed that many steps back."""
    rng = np.random.default_rng(32)
    lay = fo.Layout([6])
    p = _params(KB=2.0, KT=2.0, dt=0.1, tol=1e-10)
    st = _random_filament_state(rng, lay, p, twist=0.1)
    ext = fo.External(Fext=np.tile([0, 0, -1.0], (lay.S, 1)))
    seen = [st]
    for k in range(1, 5):
        st, _ = fo.step(lay, p, st, ext, order=2)
        seen.append(st)
        assert (st.Yprev2 is not None) == (k >= 2)
        assert (st.u_prev is not None) == (k >= 2)
        assert (st.u_prev2 is not None) == (k >= 3)
        if k >= 2:
            np.testing.assert_array_equal(st.Yprev2, seen[k - 2].Y)
            np.testing.assert_array_equal(st.u_prev, seen[k - 1].u)
            np.testing.assert_array_equal(st.lam_prev, seen[k - 1].lam)
        if k >= 3:
            np.testing.assert_array_equal(st.u_prev2, seen[k - 2].u)
            np.testing.assert_array_equal(st.lam_prev2, seen[k - 2].lam)


def test_quadratic_guess_keeps_the_solution_and_saves_iterations():
    """The converged step does not depend on X_0 beyond the tolerance: 12 steps
    of a settling, bending pair of filaments with order 1 and order 2 end at
    the same positions to within a few tolerances, and from the fourth step on
    the quadratic guess starts closer (smaller ||f(X_0)||) on every step."""
    rng = np.random.default_rng(33)
    lay = fo.Layout([8, 8])
    p = _params(KB=2.0, KT=2.0, dt=0.1, tol=1e-11)
    st0 = _random_filament_state(rng, lay, p, twist=0.05)
    st0.Y = st0.Y + np.repeat(np.array([[0.0, 0, 0], [12.0, 0, 0]]), 8, axis=0)
    ext = fo.External(Fext=np.tile([0, 0, -1.0], (lay.S, 1)), follower=np.array([0.2, 0.0]))
    sts = {1: st0, 2: st0}
    for k in range(12):
        f0 = {}
        for order in (1, 2):
            br = fo.begin_step(lay, p, sts[order], ext, order=order)
            f0[order] = np.abs(br.f).max()
            while not br.converged():
                br.iterate()
            sts[order] = fo.commit_step(lay, p, sts[order], br.X)
        if k >= 3:
            assert f0[2] < f0[1], (k, f0)
    np.testing.assert_allclose(sts[2].Y, sts[1].Y, rtol=0, atol=1e-8)


def _two_filament_history():
    """Two filaments (5 and 3 segments) whose Y_1, u and Lambda histories are
    built block by block: quadratic in the step index (x* its continuation),
    linear with alternating noise on the past values (x* the clean
    continuation), or exactly linear (x* its continuation)."""
    rng = np.random.default_rng(34)
    lay = fo.Layout([5, 3])
    first = [lay.off_seg[i] for i in range(lay.M)]

    def series(shape, kind):
        # small integer coefficients and binary-fraction noise: every
        # extrapolation below is exact in floating point, so ties are ties
        c = rng.integers(-4, 5, size=(3,) + shape).astype(np.float64)
        vals = [c[0] + c[1] * t + (c[2] * t * t if kind == "quad" else 0.0)
                for t in (1.0, 0.0, -1.0, -2.0)]          # x*, x^j, x^{j-1}, x^{j-2}
        if kind == "noisy":
            noise = 0.5 * np.abs(c[2]) + 0.25
            vals[1] = vals[1] + noise
            vals[2] = vals[2] - noise
            vals[3] = vals[3] + noise
        return vals

    return lay, first, series


def _history_state(lay, first, series, kinds):
    """State (steps=3) and solution X from per-filament (Y_1, u, Lambda) kinds."""
    Y = np.zeros((4, lay.S, 3))
    U = np.zeros((4, lay.S, 3))
    L = np.zeros((4, lay.n_lam, 3))
    for i, (ky, ku, kl) in enumerate(kinds):
        s, e = lay.off_seg[i], lay.off_seg[i + 1]
        vy = series((3,), ky)
        vu = series((e - s, 3), ku)
        vl = series((e - s - 1, 3), kl)
        for k in range(4):
            Y[k, s:e] = vy[k]
            U[k, s:e] = vu[k]
            L[k, lay.off_lam[i]:lay.off_lam[i + 1]] = vl[k]
    st = fo.State(Y=Y[1], q=np.tile([1.0, 0, 0, 0], (lay.S, 1)), Yprev=Y[2], Yprev2=Y[3],
                  u=U[1], u_prev=U[2], u_prev2=U[3], lam=L[1], lam_prev=L[2],
                  lam_prev2=L[3], steps=3)
    return st, lay.join_X(Y[0][first], U[0], L[0])


def test_adaptive_fit_of_one_commit():
    """One commit's fit: theta = 1 where the block's past is quadratic (the
    solution departs from the linear guess by exactly the second difference),
    0 where noise on the past values (+n, -n, +n) makes the second difference
    4n point against the departure -3n (the clip at 0: linear), 0 where the
    past is exactly linear (no second difference: Q = 0); per filament and
    block; no fit where three past values do not exist."""
    lay, first, series = _two_filament_history()
    st, X = _history_state(lay, first, series, [("quad", "noisy", "lin"),
                                                ("noisy", "quad", "quad")])
    fit = fo.adaptive_fit(lay, st, X)
    theta = np.array([[fo.fit_theta(fit[i, b]) for b in range(3)] for i in range(2)])
    np.testing.assert_array_equal(theta, [[1.0, 0.0, 0.0], [0.0, 1.0, 1.0]])
    assert fit[0, 2, 1] == 0.0                          # exactly linear: Q = 0
    assert fit[1, 0, 0] < 0                             # noise: P < 0, clipped
    st.u_prev2 = st.lam_prev2 = None
    fit = fo.adaptive_fit(lay, st, X)
    assert np.all(fit[:, 1:] == 0) and np.all(fit[:, 0, 1] > 0)
    st.Yprev2 = None
    assert np.all(fo.adaptive_fit(lay, st, X) == 0)


def test_adaptive_fit_is_the_weighted_least_squares_coefficient():
    """Over several commits the fit's theta minimises
    sum_k 0.7^age_k |x*_k - l_k - theta d_k|^2 (checked by a bounded scalar
    minimisation of that objective), for a block whose departures are a noisy
    fraction of its second differences."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(36)
    lay = fo.Layout([4])
    st = fo.State(Y=np.zeros((4, 3)), q=np.tile([1.0, 0, 0, 0], (4, 1)), steps=3)
    terms = []
    for k in range(6):
        hist = [rng.standard_normal((4, 3)) for _ in range(3)]
        st.u, st.u_prev, st.u_prev2 = hist
        st.Yprev, st.Yprev2 = np.zeros((4, 3)), None     # u needs Y^{j-1}; no Y_1 fit
        st.lam = st.lam_prev = st.lam_prev2 = np.zeros((3, 3))
        lin = 2 * hist[0] - hist[1]
        d = hist[0] - 2 * hist[1] + hist[2]
        xs = lin + 0.4 * d + 0.3 * rng.standard_normal((4, 3))
        X = lay.join_X(np.zeros((1, 3)), xs, np.zeros((3, 3)))
        st.xfit = fo.adaptive_fit(lay, st, X)
        terms.append((xs - lin, d))
    ages = np.arange(len(terms))[::-1]

    def objective(c):
        return sum(0.7 ** a * np.sum((r - c * d) ** 2) for a, (r, d) in zip(ages, terms))

    best = minimize_scalar(objective, bounds=(-2, 3), method="bounded",
                           options={"xatol": 1e-10}).x
    theta = fo.fit_theta(st.xfit[0, 1])
    assert 0 < theta < 1
    assert abs(theta - best) < 1e-7, (theta, best)


def test_adaptive_guess_uses_each_blocks_theta():
    """initial_guess(order=ADAPTIVE) gives each block the linear guess plus its
    theta times the second difference (quadratic histories: theta = 1 is their
    continuation, 0 the linear guess), and with no fit the linear guess."""
    lay, first, series = _two_filament_history()
    vy = series((lay.S, 3), "quad")
    vu = series((lay.S, 3), "quad")
    vl = series((lay.n_lam, 3), "quad")
    thetas = np.array([[1.0, 0.25, 0.0], [0.5, 1.0, 0.75]])
    fit = np.stack([thetas * 2.0, np.full((2, 3), 2.0)], axis=-1)     # P = 2 theta, Q = 2
    st = fo.State(Y=vy[1], q=np.tile([1.0, 0, 0, 0], (lay.S, 1)), Yprev=vy[2], Yprev2=vy[3],
                  u=vu[1], u_prev=vu[2], u_prev2=vu[3], lam=vl[1], lam_prev=vl[2],
                  lam_prev2=vl[3], steps=3, xfit=fit)
    X0 = fo.initial_guess(lay, st, order=fo.ADAPTIVE)
    Y1, u, lam = lay.split_X(X0)
    blocks = ((Y1, [x[first] for x in vy], lambda i: slice(i, i + 1)),
              (u, vu, lambda i: slice(lay.off_seg[i], lay.off_seg[i + 1])),
              (lam, vl, lambda i: slice(lay.off_lam[i], lay.off_lam[i + 1])))
    for b, (got, v, rows_of) in enumerate(blocks):
        for i in range(lay.M):
            r = rows_of(i)
            lin = 2 * v[1][r] - v[2][r]
            want = lin + thetas[i, b] * (v[0][r] - lin)       # v[0] - lin = d for these
            np.testing.assert_allclose(got[r], want, rtol=0, atol=1e-12)
    st.xfit = None
    np.testing.assert_allclose(fo.initial_guess(lay, st, order=fo.ADAPTIVE),
                               fo.initial_guess(lay, st, order=1), rtol=0, atol=0)


def test_adaptive_guess_keeps_the_solution():
    """Adaptive and linear runs of the same 12 steps end at the same
    positions to within a few tolerances, and the adaptive run takes no more
    Broyden iterations in all."""
    rng = np.random.default_rng(35)
    lay = fo.Layout([8, 8])
    p = _params(KB=2.0, KT=2.0, dt=0.1, tol=1e-9)
    st0 = _random_filament_state(rng, lay, p, twist=0.05)
    st0.Y = st0.Y + np.repeat(np.array([[0.0, 0, 0], [12.0, 0, 0]]), 8, axis=0)
    ext = fo.External(Fext=np.tile([0, 0, -1.0], (lay.S, 1)), follower=np.array([0.2, 0.0]))
    end, its = {}, {}
    for order in (1, fo.ADAPTIVE):
        st, n = st0, 0
        for _ in range(12):
            st, k = fo.step(lay, p, st, ext, order=order)
            n += k
        end[order], its[order] = st.Y, n
    np.testing.assert_allclose(end[fo.ADAPTIVE], end[1], rtol=0, atol=1e-7)
    assert its[fo.ADAPTIVE] <= its[1], its


# --------------------------------------------------------------------------
# Broyden memory carried across steps (an option; the paper resets H_0 = J0^{-1})
# --------------------------------------------------------------------------

def _carry_system(seed):
    rng = np.random.default_rng(seed)
    lay = fo.Layout([8, 8, 8])
    p = _params(KB=2.0, KT=2.0, dt=0.2, tol=1e-11)
    st = _random_filament_state(rng, lay, p, twist=0.05)
    st.Y = st.Y + np.repeat(np.array([[0.0, 0, 0], [9.0, 0, 0], [0, 9.0, 0]]), 8, axis=0)
    ext = fo.External(Fext=np.tile([0, 0, -1.5], (lay.S, 1)), follower=np.array([0.3, 0.0, 0.1]))
    return lay, p, st, ext


def test_carried_memory_starts_from_the_previous_inverse():
    """With every pair of a converged step carried and its J0 kept, the next
    step's H_0 is the previous step's final H: it satisfies that step's last
    secant equation H dF = dX (bad Broyden's H_{k+1} does) to rounding, more
    than a thousand times closer than J0^{-1} alone."""
    lay, p, st, ext = _carry_system(40)
    st, _ = fo.step(lay, p, st, ext, j0_model="rpy")            # a BDF2 history
    br = fo.begin_step(lay, p, st, ext, j0_model="rpy")
    Xs, fs = [br.X.copy()], [br.f.copy()]
    while not br.converged():
        br.iterate()
        Xs.append(br.X.copy())
        fs.append(br.f.copy())
    assert br.k >= 3
    dX, dF = Xs[-1] - Xs[-2], fs[-1] - fs[-2]
    st2 = fo.commit_step(lay, p, st, br.X)
    nxt = fo.begin_step(lay, p, st2, ext, j0=br.solver, memory=list(zip(br.c, br.d)))
    err_h = np.abs(nxt.H(dF) - dX).max()
    err_j0 = np.abs(br.solver.solve(dF) - dX).max()
    assert err_h <= 1e-14 * np.abs(br.X).max() and err_h < 1e-3 * err_j0, (err_h, err_j0)


def test_carried_memory_keeps_the_solution():
    """Eight steps with J0 kept and the previous step's pairs carried (at most
    12, the most recent) against the same steps with H_0 = J0^{-1}: the same
    positions to within a few tolerances. (Whether it saves iterations depends
    on how much coupling between filaments J0 leaves out: here, three distant
    filaments, it does not; on large clouds it does.)"""
    lay, p, st0, ext = _carry_system(41)
    st0, _ = fo.step(lay, p, st0, ext, j0_model="rpy")
    ends, its = {}, {}
    for keep in (0, 12):
        st, solver, mem, n = st0, None, [], 0
        for j in range(8):
            br = fo.begin_step(lay, p, st, ext, j0_model="rpy", j0=solver,
                               memory=mem[-keep:] if keep else ())
            while not br.converged():
                br.iterate()
                n += 1
            solver, mem = br.solver, list(zip(br.c, br.d))
            st = fo.commit_step(lay, p, st, br.X)
        ends[keep], its[keep] = st.Y, n
    np.testing.assert_allclose(ends[12], ends[0], rtol=0, atol=1e-8)
    assert its[12] > 8 and its[0] > 8, its


def test_adaptive_fit_skips_a_step_without_iterations():
    """A commit whose solution is the guess itself (no Broyden iteration)
    leaves the fit as it was; the same commit counted as iterated moves it."""
    lay, first, series = _two_filament_history()
    st, X = _history_state(lay, first, series, [("quad", "noisy", "quad"),
                                                ("noisy", "quad", "noisy")])
    st.xfit = np.full((lay.M, 3, 2), 0.5)
    st.q = fo.qmul(fo.qexp(np.zeros((lay.S, 3))), st.q)
    p = _params()
    kept = fo.commit_step(lay, p, st, X, order=fo.ADAPTIVE, iterated=False)
    np.testing.assert_array_equal(kept.xfit, st.xfit)
    moved = fo.commit_step(lay, p, st, X, order=fo.ADAPTIVE, iterated=True)
    assert np.abs(moved.xfit - st.xfit).max() > 0.1
