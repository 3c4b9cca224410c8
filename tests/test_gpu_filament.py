"""GPU parity of the residual, J0 solve, Broyden iterates and timesteps
(fil_residual, fil_j0_solve, fil_broyden_*, fil_step, fil_init_straight)
against the oracle, plus the error statuses.

FP64 path tolerances: residual entries within 1e-12 of the oracle relative to
the largest position magnitude (the rows subtract O(|Y|) terms); J0 solves and
Broyden iterates within 1e-10 relative (they go through a pivoted banded LU on
the GPU and a dense LU in the oracle, whose rounding differs by cond(J0) eps).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filament as fo  # noqa: E402
from paper_1903_12609_gb300.inputs import (random_frames, single_filament,  # noqa: E402
                                           suspension, workload_params)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


def _system(segs, seed, history=False, KB=2.0, KT=1.5, dt=0.1, tol=1e-10, twist=0.05,
            follower=True, **extra):
    rng = np.random.default_rng(seed)
    lay = fo.Layout(segs)
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=KB, KT=KT, dt=dt, tol=tol, max_iter=60, **extra)
    M = len(segs)
    base = rng.uniform(0, 6.0 * M ** (1 / 3) * 3, size=(M, 3))
    t, mu = random_frames(rng, M)
    xi = twist * rng.standard_normal((lay.S, 3))
    st = fo.initial_state(lay, p, base, t, mu, xi)
    if history:
        st.Yprev = st.Y + 0.01 * rng.standard_normal(st.Y.shape)
        st.u = 0.02 * rng.standard_normal((lay.S, 3))
    st.lam = 0.1 * rng.standard_normal((lay.n_lam, 3))
    ext = fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1)),
                      Text=0.05 * rng.standard_normal((lay.S, 3)),
                      follower=(rng.uniform(0, 1, M) if follower else None))
    return lay, p, st, ext, (base, t, mu, xi)


def _gpu(fil, lay, p, st, ext, prec=0, j0=0):
    m = fil.Filaments(lay.N, a=p.a, eta=p.eta, dL=p.dL, KB=p.KB, KT=p.KT, gamma0=p.gamma0,
                      kappa_mu=p.kappa_mu, kappa_nu=p.kappa_nu, dt=p.dt, tol=p.tol,
                      max_iter=p.max_iter, precision=prec, j0_model=j0)
    m.set_state(st.Y, st.q, st.Yprev, st.u, st.lam if lay.n_lam else None)
    m.set_external(ext.Fext, ext.Text, ext.follower)
    return m


SEGS = [[20], [1, 5, 33], [32] * 6, [40, 65, 2, 1]]


def test_full_size_residual_on_sampled_filaments(fil):
    """The 32 000-segment suspension (1000 x 32, its physics and external loads),
    FP64 path: the residual rows of sampled filaments against the oracle. The
    oracle evaluates the mobility on those filaments' rows only (sources: all
    32 000 segments); everything else it computes for the whole system."""
    from oracle import rpy
    wl, base, t, mu, Fext, follower = suspension(1000, 32, seed=0)
    lay = fo.Layout([32] * 1000)
    p = fo.Params(a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                  max_iter=wl.max_iter)
    st = fo.initial_state(lay, p, base, t, mu)
    ext = fo.External(Fext=Fext, follower=follower)
    rng = np.random.default_rng(7)
    X = fo.initial_guess(lay, st)
    X = X + 1e-3 * rng.standard_normal(X.shape)
    fils = [0, 1, 499, 500, 998, 999] + list(rng.choice(np.arange(2, 998), 6, replace=False))
    rows = np.concatenate([np.arange(32 * i, 32 * i + 32) for i in fils]).astype(np.int32)

    def sampled_mobility(Y, F, T, p, nthreads=1):
        V = np.zeros_like(Y)
        W = np.zeros_like(Y)
        VW = rpy.apply_rows(Y, np.concatenate([F, T], axis=1), rows, p.a, p.eta, nthreads=8)
        V[rows], W[rows] = VW[:, :3], VW[:, 3:]
        return V, W

    ref = fo.residual(lay, p, st, ext, X, mob=sampled_mobility)
    with _gpu(fil, lay, p, st, ext) as m:
        f = np.zeros(6 * lay.S)
        m.residual(X, f)
    scale = max(1.0, np.abs(st.Y).max())
    for i in fils:
        b = lay.off_X[i]
        np.testing.assert_allclose(f[b:b + 6 * 32], ref[b:b + 6 * 32], rtol=0, atol=1e-12 * scale)


def _subsystem(lay, st, X, fils):
    """The filaments `fils` of a system as a system of their own (state and X
    sliced; per-filament quantities such as J0 blocks do not depend on the rest)."""
    sub = fo.Layout([lay.N[i] for i in fils])
    seg = np.concatenate([np.arange(lay.off_seg[i], lay.off_seg[i] + lay.N[i]) for i in fils])
    lam_rows = np.concatenate([np.arange(lay.off_seg[i] - i, lay.off_seg[i] - i + lay.N[i] - 1)
                               for i in fils])
    xs = np.concatenate([X[lay.off_X[i]:lay.off_X[i] + 6 * lay.N[i]] for i in fils])

    def cut(a, rows):
        return None if a is None else a[rows].copy()
    st_sub = fo.State(Y=st.Y[seg].copy(), q=st.q[seg].copy(), Yprev=cut(st.Yprev, seg),
                      u=cut(st.u, seg), lam=cut(st.lam, lam_rows), steps=st.steps)
    return sub, st_sub, xs


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_full_size_j0_solve_on_sampled_filaments(fil, prec):
    """The 32 000-segment suspension with the filament-RPY J0 (the bench's
    configuration): J0^{-1} b on sampled filaments against the oracle's dense
    LU of the same blocks, FP64 path (and FIL_PAIR32, whose J0 solves are the
    FP64 path's) to 1e-10. The FIL_MIXED path assembles and
    inverts J0 in FP32 with no refinement; its normwise backward error against
    the oracle's blocks, |B x - b|_inf / (|B|_inf |x|_inf + |b|_inf) per block,
    is bounded by 2 n u_32 (n = 6N = 192: an FP32 Gauss-Jordan inverse, and an
    assembly whose entries sum at most n products), independent of cond(B)."""
    wl, base, t, mu, Fext, follower = suspension(1000, 32, seed=0)
    lay = fo.Layout([32] * 1000)
    p = fo.Params(a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                  max_iter=wl.max_iter)
    st = fo.initial_state(lay, p, base, t, mu)
    ext = fo.External(Fext=Fext, follower=follower)
    rng = np.random.default_rng(8)
    fils = [0, 999] + list(rng.choice(np.arange(1, 999), 6, replace=False))
    b = rng.standard_normal(6 * lay.S)
    with _gpu(fil, lay, p, st, ext, prec=prec, j0=1) as m:
        m.broyden_begin()
        X0 = np.zeros(6 * lay.S)
        m.get_iterate(X0, None)
        x = np.zeros_like(b)
        m.j0_solve(b, x)
    np.testing.assert_allclose(X0, fo.initial_guess(lay, st), rtol=0, atol=1e-12)
    sub, st_sub, X0_sub = _subsystem(lay, st, X0, fils)
    blocks = fo.jacobian0_general(sub, p, st_sub, X0_sub, "rpy")
    b_sub = np.concatenate([b[lay.off_X[i]:lay.off_X[i] + 192] for i in fils])
    ref = fo.J0Solver(sub, blocks).solve(b_sub)
    got = np.concatenate([x[lay.off_X[i]:lay.off_X[i] + 192] for i in fils])
    if prec != fil.FIL_MIXED:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    else:
        u32 = 2.0 ** -24
        for B, o in zip(blocks, sub.off_X):
            xi, bi = got[o:o + 192], b_sub[o:o + 192]
            eta = np.abs(B @ xi - bi).max() / (np.abs(B).sum(axis=1).max() * np.abs(xi).max()
                                                + np.abs(bi).max())
            assert eta <= 2 * 192 * u32, eta


@pytest.mark.parametrize("segs", SEGS)
@pytest.mark.parametrize("history", [False, True])
def test_residual_parity(fil, segs, history):
    lay, p, st, ext, _ = _system(segs, 10 + len(segs), history=history, gamma0=0.1,
                                 kappa_mu=-0.05, kappa_nu=0.2)
    rng = np.random.default_rng(1)
    Y1 = np.array([st.Y[lay.off_seg[i]] for i in range(lay.M)]) + 0.01
    X = lay.join_X(Y1, 0.05 * rng.standard_normal((lay.S, 3)),
                   rng.standard_normal((lay.n_lam, 3)))
    ref = fo.residual(lay, p, st, ext, X, nthreads=4)
    with _gpu(fil, lay, p, st, ext) as m:
        f = np.zeros(6 * lay.S)
        finf = m.residual(X, f)
    scale = max(1.0, np.abs(st.Y).max())
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-12 * scale)
    assert abs(finf - np.abs(f).max()) == 0.0


@pytest.mark.parametrize("prec", [1, 2])
def test_residual_mixed_close_to_fp64(fil, prec):
    lay, p, st, ext, _ = _system([32] * 6, 3, history=True)
    X = fo.initial_guess(lay, st)
    ref = fo.residual(lay, p, st, ext, X)
    with _gpu(fil, lay, p, st, ext, prec=prec) as m:
        f = np.zeros(6 * lay.S)
        m.residual(X, f)
    # velocity errors of a few 1e-7 relative, times (2/3) dt
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("segs", SEGS)
def test_init_straight_matches_oracle(fil, segs):
    lay, p, st, ext, (base, t, mu, xi) = _system(segs, 20)
    with _gpu(fil, lay, p, st, ext) as m:
        m.init_straight(base, t, mu, xi)
        Y = np.zeros((lay.S, 3))
        q = np.zeros((lay.S, 4))
        m.get_state(Y, q, None, None, None)
    np.testing.assert_allclose(Y, st.Y, rtol=0, atol=1e-12 * max(1, np.abs(st.Y).max()))
    np.testing.assert_allclose(q, st.q, rtol=0, atol=1e-14)


J0_MODELS = [(0, "drag"), (1, "rpy")]


@pytest.mark.parametrize("segs", SEGS[:3] + [[38, 2, 1], [40, 65, 2, 1]])
@pytest.mark.parametrize("history", [False, True])
@pytest.mark.parametrize("model", J0_MODELS)
@pytest.mark.parametrize("prec", [0, 2])
def test_j0_solve_matches_dense_oracle(fil, segs, history, model, prec):
    """FP64 J0 solves (FIL_FP64, and FIL_PAIR32 whose J0 is the same) against the
    oracle's dense LU of App. B.2's blocks or the filament-RPY blocks."""
    if model[0] == 1 and max(segs) > 38:
        pytest.skip("the filament-RPY J0 supports N <= 38 segments per filament")
    lay, p, st, ext, _ = _system(segs, 30, history=history, twist=0.2)
    with _gpu(fil, lay, p, st, ext, prec=prec, j0=model[0]) as m:
        m.broyden_begin()
        X0 = np.zeros(6 * lay.S)
        m.get_iterate(X0, None)
        np.testing.assert_allclose(X0, fo.initial_guess(lay, st), rtol=0, atol=1e-14 * 100)
        b = np.random.default_rng(2).standard_normal(6 * lay.S)
        x = np.zeros_like(b)
        m.j0_solve(b, x)
    blocks = (fo.jacobian0(lay, p, st, X0) if model[1] == "drag"
              else fo.jacobian0_general(lay, p, st, X0, model[1]))
    ref = fo.J0Solver(lay, blocks).solve(b)
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("segs", [[20], [32] * 6, [1, 7, 32, 13], [33, 3]])
def test_mixed_j0_solve_within_fp32_rounding(fil, segs):
    """Mixed mode applies an FP32 Gauss-Jordan inverse of each filament-RPY block
    without refinement (a register kernel for 6N <= 192, a shared-memory one
    above). Its error is bounded by that of an FP32 dense LU solve of the same
    blocks, the rounding the arithmetic allows, times a small factor; an index or
    pivoting mistake would be O(1)."""
    lay, p, st, ext, _ = _system(segs, 31, history=True, twist=0.2)
    with _gpu(fil, lay, p, st, ext, prec=fil.FIL_MIXED, j0=1) as m:
        m.broyden_begin()
        X0 = np.zeros(6 * lay.S)
        m.get_iterate(X0, None)
        b = np.random.default_rng(3).standard_normal(6 * lay.S)
        x = np.zeros_like(b)
        m.j0_solve(b, x)
    blocks = fo.jacobian0_general(lay, p, st, X0, "rpy")
    ref = fo.J0Solver(lay, blocks).solve(b)
    x32 = np.concatenate([np.linalg.solve(B.astype(np.float32), b[o:o + B.shape[0]].astype(
        np.float32)).astype(np.float64) for B, o in zip(blocks, lay.off_X)])
    e32 = np.abs(x32 - ref).max()
    assert e32 < 1e-3 * np.abs(ref).max()
    assert np.abs(x - ref).max() <= 16 * e32 + 1e-12


@pytest.mark.parametrize("segs", [[20], [32] * 4, [1, 7, 33]])
@pytest.mark.parametrize("model", J0_MODELS)
def test_broyden_iterates_match_oracle(fil, segs, model):
    lay, p, st, ext, _ = _system(segs, 40, history=True, tol=1e-13)
    br = fo.begin_step(lay, p, st, ext, j0_model=model[1])
    with _gpu(fil, lay, p, st, ext, j0=model[0]) as m:
        f0 = m.broyden_begin()
        assert abs(f0 - np.abs(br.f).max()) <= 1e-12 * max(1, np.abs(st.Y).max())
        X = np.zeros(6 * lay.S)
        f = np.zeros(6 * lay.S)
        for k in range(6):
            conv, finf = m.broyden_step()
            br.iterate()
            m.get_iterate(X, f)
            sc = np.abs(br.X).max()
            np.testing.assert_allclose(X, br.X, rtol=0, atol=1e-10 * sc)
            np.testing.assert_allclose(f, br.f, rtol=0, atol=1e-10 * max(1, np.abs(br.f).max()))
            if conv:
                break


def test_c0_trajectory_parity(fil):
    """Single tilted filament, N = 20, B = 1000, dt = T/100, tol 1e-8: 200 steps,
    positions within 1e-8 over the first 25 steps and 1e-6 over all of them."""
    wl = workload_params(1, 20, B=1000.0, dt_over_T=0.01, tol=1e-8)
    base, t, mu, xi = single_filament(20, seed=0)
    lay = fo.Layout([20])
    p = fo.Params(a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                  max_iter=50)
    st = fo.initial_state(lay, p, base, t, mu, xi)
    ext = fo.External(Fext=np.tile([0.0, 0.0, -wl.W * wl.dL], (20, 1)))
    with _gpu(fil, lay, p, st, ext) as m:
        m.init_straight(base, t, mu, xi)
        Y = np.zeros((20, 3))
        q = np.zeros((20, 4))
        for j in range(200):
            st, it_ref = fo.step(lay, p, st, ext)
            it = m.step()
            m.get_state(Y, q, None, None, None)
            assert abs(it - it_ref) <= 1
            np.testing.assert_allclose(Y, st.Y, rtol=0, atol=1e-8 if j < 25 else 1e-6)
            np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_step_converges_close_to_fp64(fil, prec):
    lay, p, st, ext, _ = _system([32] * 8, 50, tol=1e-6, dt=0.2)
    ref = st
    for _ in range(3):
        ref, _ = fo.step(lay, p, ref, ext)
    with _gpu(fil, lay, p, st, ext, prec=prec) as m:
        for _ in range(3):
            m.step()
        Y = np.zeros((lay.S, 3))
        m.get_state(Y, None, None, None, None)
    np.testing.assert_allclose(Y, ref.Y, rtol=0, atol=1e-4)


def test_error_statuses(fil):
    lay, p, st, ext, _ = _system([10, 10], 60)
    with _gpu(fil, lay, p, st, ext) as m:
        with pytest.raises(fil.FilError) as e:
            m.broyden_step()
        assert e.value.status == fil.FIL_ESTATE
        with pytest.raises(fil.FilError) as e:
            m.broyden_commit()
        assert e.value.status == fil.FIL_ESTATE
        bad = st.Y.copy()
        bad[3, 1] = np.nan
        m.set_state(bad, st.q)
        with pytest.raises(fil.FilError) as e:
            m.step()
        assert e.value.status == fil.FIL_ENAN
    # max_iter = 1 on a stiff step cannot converge to 1e-14
    p1 = fo.Params(**{**p.__dict__, "max_iter": 1, "tol": 1e-14, "dt": 1.0})
    with _gpu(fil, lay, p1, st, ext) as m:
        Y0 = np.zeros((lay.S, 3))
        m.get_state(Y0, None, None, None, None)
        with pytest.raises(fil.FilError) as e:
            m.step()
        assert e.value.status == fil.FIL_ENOCONV
        Y1 = np.zeros((lay.S, 3))
        m.get_state(Y1, None, None, None, None)
        np.testing.assert_array_equal(Y0, Y1)       # state untouched on failure


def test_filament_rpy_j0_step_matches_oracle(fil):
    """Timesteps with the filament-RPY J0 agree with the oracle driven the same way."""
    lay, p, st, ext, _ = _system([32] * 5, 70, tol=1e-10, dt=0.3)
    with _gpu(fil, lay, p, st, ext, j0=1) as m:
        Y = np.zeros((lay.S, 3))
        for _ in range(3):
            st, it_ref = fo.step(lay, p, st, ext, j0_model="rpy")
            it = m.step()
            assert abs(it - it_ref) <= 1
            m.get_state(Y, None, None, None, None)
            np.testing.assert_allclose(Y, st.Y, rtol=0, atol=1e-8)


def test_filament_rpy_j0_rejects_long_filaments(fil):
    with pytest.raises(fil.FilError) as e:
        fil.Filaments([39], j0_model=1)
    assert e.value.status == fil.FIL_EINVAL


def test_bdf2_second_order_in_time_on_gpu(fil):
    """Sec. 4.2's 3D test on the GPU: four vertical filaments of N = 30 at the
    corners of a square of side 0.268 L, B = 1000, settling for 2T; the maximum
    position error against dt = T/1600 falls by ~4 per halving of dt."""
    N = 30
    wl = workload_params(4, N, B=1000.0, dt_over_T=0.01, tol=1e-10)
    T = wl.extra["T"]
    D = 0.268 * wl.extra["L"]
    base = np.array([[0, 0, 0], [D, 0, 0], [0, D, 0], [D, D, 0]], dtype=float)
    lay = fo.Layout([N] * 4)
    Fext = np.tile([0.0, 0.0, -wl.W * wl.dL], (lay.S, 1))

    def run(n_steps):
        with fil.Filaments(lay.N, a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT,
                           dt=2.0 * T / n_steps, tol=wl.tol, max_iter=100) as m:
            m.init_straight(base, np.tile([0.0, 0.0, 1.0], (4, 1)),
                            np.tile([1.0, 0.0, 0.0], (4, 1)), None)
            m.set_external(Fext, None, None)
            for _ in range(n_steps):
                m.step()
            Y = np.zeros((lay.S, 3))
            m.get_state(Y, None, None, None, None)
            return Y

    ref = run(3200)
    err = [np.linalg.norm(run(n) - ref, axis=1).max() for n in (50, 100, 200)]
    assert 3.5 < err[0] / err[1] < 4.5, err
    assert 3.5 < err[1] / err[2] < 4.5, err


@pytest.mark.parametrize("unorm", [1e-9, 0.01, 0.2499, 0.2501, 0.8])
def test_residual_parity_across_small_angle_branches(fil, unorm):
    """Rotation vectors on both sides of |u| = 1/4, where the quaternion exponential and the
    dexpinv coefficient switch from their series to sincos / tan: the residual (which uses
    both) matches the oracle to the FP64 tolerance."""
    lay, p, st, ext, _ = _system([12, 7], 77, history=True)
    rng = np.random.default_rng(3)
    d = rng.standard_normal((lay.S, 3))
    u = unorm * d / np.linalg.norm(d, axis=1, keepdims=True)
    Y1 = np.array([st.Y[lay.off_seg[i]] for i in range(lay.M)])
    X = lay.join_X(Y1, u, rng.standard_normal((lay.n_lam, 3)))
    ref = fo.residual(lay, p, st, ext, X)
    with _gpu(fil, lay, p, st, ext) as m:
        f = np.zeros(6 * lay.S)
        m.residual(X, f)
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(st.Y).max()))


@pytest.mark.parametrize("model", J0_MODELS)
def test_j0_reuse_keeps_the_converged_trajectory(fil, model):
    """J0 only shapes the iterates of Algorithm 2: with the factors of one step
    reused for up to 4 steps (fil_set_j0_reuse) every step still converges to
    ||f||_inf <= tol a, and the trajectory stays on the oracle's (which builds J0
    every step) to within the tolerance the iterates are solved to."""
    lay, p, st, ext, _ = _system([32] * 5, 71, tol=1e-10, dt=0.3)
    with _gpu(fil, lay, p, st, ext, j0=model[0]) as m:
        m.set_j0_reuse(4)
        Y = np.zeros((lay.S, 3))
        for _ in range(8):
            st, _ = fo.step(lay, p, st, ext, j0_model=model[1])
            m.step()
            m.get_state(Y, None, None, None, None)
            np.testing.assert_allclose(Y, st.Y, rtol=0, atol=1e-8)
        builds, reuses = m.j0_stats()
        assert builds + reuses == 8 and reuses >= 3, (builds, reuses)
        # a new state invalidates the factors: the next step builds J0
        m.set_state(st.Y, st.q)
        m.step()
        assert m.j0_stats()[0] == builds + 1


def test_j0_reuse_off_and_argument_checks(fil):
    lay, p, st, ext, _ = _system([16] * 3, 72, tol=1e-10, dt=0.3)
    with _gpu(fil, lay, p, st, ext) as m:
        for _ in range(3):
            m.step()
        assert m.j0_stats() == (3, 0)           # the default builds J0 every step
        with pytest.raises(fil.FilError) as e:
            m.set_j0_reuse(0)
        assert e.value.status == fil.FIL_EINVAL
        m.broyden_begin()
        with pytest.raises(fil.FilError) as e:
            m.set_j0_reuse(3)
        assert e.value.status == fil.FIL_ESTATE


@pytest.mark.parametrize("history", [False, True])
@pytest.mark.parametrize("model", J0_MODELS)
def test_quadratic_extrapolation_matches_oracle(fil, history, model):
    """fil_set_extrapolation(2): X_0 of each of 7 steps equals the oracle's
    order-2 guess (the oracle stepping alongside at the same tolerance; X_0
    inherits the two trajectories' difference, within a few tolerances, times
    the extrapolation weights 3 + 3 + 1), and it is not the linear guess once
    three committed values exist. With Y^{j-1} given to fil_set_state, Y_1 is
    quadratic from the second step on; u and Lambda from the fourth."""
    lay, p, st, ext, _ = _system([20, 7, 33], 73, history=history, tol=1e-12, dt=0.2)
    with _gpu(fil, lay, p, st, ext, j0=model[0]) as m:
        assert m.extrapolation() == 1
        m.set_extrapolation(2)
        assert m.extrapolation() == 2
        X0 = np.zeros(6 * lay.S)
        for k in range(7):
            br = fo.begin_step(lay, p, st, ext, j0_model=model[1], order=2)
            m.broyden_begin()
            m.get_iterate(X0, None)
            sc = max(1.0, np.abs(br.X).max())
            np.testing.assert_allclose(X0, br.X, rtol=0, atol=1e-9 * sc)
            if k >= 3:
                lin = fo.initial_guess(lay, st, order=1)
                assert np.abs(lin - br.X).max() > 1e3 * 1e-9 * sc
            while True:
                conv, _ = m.broyden_step()
                if conv:
                    break
            m.broyden_commit()
            while not br.converged():
                br.iterate()
            st = fo.commit_step(lay, p, st, br.X)


def test_extrapolation_argument_checks(fil):
    lay, p, st, ext, _ = _system([16] * 2, 74, tol=1e-10)
    with _gpu(fil, lay, p, st, ext) as m:
        for bad in (0, 4, -1):
            with pytest.raises(fil.FilError) as e:
                m.set_extrapolation(bad)
            assert e.value.status == fil.FIL_EINVAL
        m.broyden_begin()
        with pytest.raises(fil.FilError) as e:
            m.set_extrapolation(2)
        assert e.value.status == fil.FIL_ESTATE
        assert m.extrapolation() == 1


@pytest.mark.parametrize("model", J0_MODELS)
def test_adaptive_extrapolation_matches_oracle(fil, model):
    """FIL_EXTRAP_ADAPTIVE: X_0 of each of 9 steps equals the oracle's (FP64,
    the oracle stepping alongside). The tolerance is loose (1e-6) so that the
    converged history carries noise and the fitted theta spreads over [0, 1]
    (a filament sedimenting fast, one slowly, two unforced): blocks near the
    quadratic guess, near the linear one and in between all occur. With the
    same iterations on both sides the FP64 trajectories agree to rounding, far
    inside the spread of the guesses, so a wrong fit or blend shows."""
    segs = [12, 7, 16, 9]
    rng = np.random.default_rng(75)
    lay = fo.Layout(segs)
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.2, tol=1e-6, max_iter=60)
    base = np.array([[0, 0, 0], [40.0, 0, 0], [0, 40.0, 0], [40, 40, 0]])
    t, mu = random_frames(rng, len(segs))
    st = fo.initial_state(lay, p, base, t, mu, 0.05 * rng.standard_normal((lay.S, 3)))
    F = np.zeros((lay.S, 3))
    F[lay.off_seg[0]:lay.off_seg[1], 2] = -2.0
    F[lay.off_seg[2]:lay.off_seg[3], 2] = -0.5
    ext = fo.External(Fext=F, Text=np.zeros((lay.S, 3)), follower=np.array([0.0, 0.0, 0.0, 0.3]))
    thetas = []
    with _gpu(fil, lay, p, st, ext, j0=model[0]) as m:
        m.set_extrapolation(fil.FIL_EXTRAP_ADAPTIVE)
        assert m.extrapolation() == fil.FIL_EXTRAP_ADAPTIVE
        X0 = np.zeros(6 * lay.S)
        for k in range(9):
            br = fo.begin_step(lay, p, st, ext, j0_model=model[1], order=fo.ADAPTIVE)
            conv = m.broyden_begin() <= p.tol * p.a
            m.get_iterate(X0, None)
            sc = max(1.0, np.abs(br.X).max())
            np.testing.assert_allclose(X0, br.X, rtol=0, atol=1e-9 * sc)
            n = 0
            while not conv:
                conv, _ = m.broyden_step()
                n += 1
            m.broyden_commit()
            while not br.converged():
                br.iterate()
            assert n == br.k, (k, n, br.k)
            st = fo.commit_step(lay, p, st, br.X, order=fo.ADAPTIVE, iterated=br.k > 0)
            thetas += [fo.fit_theta(pq) for pq in st.xfit.reshape(-1, 2) if pq[1] > 0]
    th = np.array(thetas)
    assert (th < 0.4).any() and (th > 0.9).any() and ((th > 0.05) & (th < 0.95)).any(), th


@pytest.mark.parametrize("model", J0_MODELS)
@pytest.mark.parametrize("tol,n_steps", [(1e-6, 6), (3e-3, 10)])
def test_carried_broyden_memory_matches_oracle(fil, model, tol, n_steps):
    """fil_set_broyden_memory(6) with J0 kept across steps: every Broyden iterate
    of n_steps steps equals the oracle's (FP64), the oracle starting each step
    from the J0 the library used (rebuilt where fil_j0_stats says it was) and
    from the last 6 of the previous step's pairs; the library skips the update
    of the iteration that converges, so that pair is not carried, and a step
    that converges on entry (H_k = H_0) passes on the pairs it carried. The
    same iteration counts, iterates within 1e-8 relative: a carried pair
    d = df / |df| from the end of a converged step has |df| ~ tol, so the two
    sides' ~1e-13 residual rounding differs in it by ~1e-13 / tol, and the
    carried steps' iterates inherit that (measured: <= 7e-10 at tol 1e-6,
    7e-7 at 1e-8, 3e-5 at 1e-11; without carried pairs 5e-13 at every tol).
    At tol 3e-3 the oracle's run has steps 5-8 converge on entry and step 9
    iterate from the 3 pairs they passed on."""
    keep = 6
    lay, p, st, ext, _ = _system([20, 32, 11], 76, history=True, tol=tol, dt=0.15)
    with _gpu(fil, lay, p, st, ext, j0=model[0]) as m:
        m.set_j0_reuse(50)
        m.set_broyden_memory(keep)
        solver, mem = None, []
        X = np.zeros(6 * lay.S)
        f = np.zeros(6 * lay.S)
        carried = 0
        held = through_hold = False   # pairs passed on by a step converged on entry
        for j in range(n_steps):
            builds = m.j0_stats()[0]
            f0 = m.broyden_begin()
            rebuilt = m.j0_stats()[0] > builds
            if rebuilt:
                solver, mem = None, []
            br = fo.begin_step(lay, p, st, ext, j0_model=model[1], j0=solver,
                               memory=mem[-keep:])
            carried += 0 if rebuilt else len(mem[-keep:])
            if rebuilt:
                held = False
            assert abs(f0 - np.abs(br.f).max()) <= 1e-12 * max(1, np.abs(st.Y).max())
            conv = f0 <= p.tol * p.a
            while not conv:
                conv, _ = m.broyden_step()
                br.iterate()
                m.get_iterate(X, f)
                sc = np.abs(br.X).max()
                np.testing.assert_allclose(X, br.X, rtol=0, atol=1e-8 * sc)
                assert conv == br.converged(), (j, br.k)
            m.broyden_commit()
            solver = br.solver
            if br.k > 0:
                through_hold = through_hold or (held and len(mem[-keep:]) > 0)
                mem = list(zip(br.c, br.d))[:-1]
                held = False
            elif mem:
                held = True
            st = fo.commit_step(lay, p, st, br.X)
        assert carried > 0, "no step started from carried pairs"
        if tol > 1e-4:
            assert through_hold, "no step iterated from pairs passed on by a converged step"


def test_broyden_memory_argument_checks(fil):
    lay, p, st, ext, _ = _system([16] * 2, 77, tol=1e-10)
    with _gpu(fil, lay, p, st, ext) as m:
        for bad in (-1, p.max_iter + 1):
            with pytest.raises(fil.FilError) as e:
                m.set_broyden_memory(bad)
            assert e.value.status == fil.FIL_EINVAL
        m.set_broyden_memory(3)
        m.broyden_begin()
        with pytest.raises(fil.FilError) as e:
            m.set_broyden_memory(2)
        assert e.value.status == fil.FIL_ESTATE
