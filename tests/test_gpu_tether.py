"""GPU parity of tethered and clamped filaments (Sec. 5.2.1; fil_set_tether)
against the oracle: residuals with multipliers in the slots, J0 solves (free
J0 plus the rank-6 correction on the GPU, dense LU of the substituted J0 in
the oracle), Broyden iterates, motor-driven steps with the multipliers, an
ensemble with tethered filaments (with and without CUDA graphs), and the
clamped elastica of Sec. 4.1 reached on the GPU.

Tolerances as for free filaments: residual entries 1e-12 of the largest
position, J0 solves and iterates 1e-10 relative, positions after steps 1e-8.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import elastica  # noqa: E402
from oracle import filament as fo  # noqa: E402
from paper_1903_12609_gb300.inputs import random_frames  # noqa: E402

pytestmark = pytest.mark.gpu

J0_MODELS = [(0, "drag"), (1, "rpy")]


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


def _gpu(fil, lay, p, st, ext, teth, prec=0, j0=0, fil_per_sys=None):
    m = fil.Filaments(lay.N, fil_per_sys=fil_per_sys, a=p.a, eta=p.eta, dL=p.dL, KB=p.KB,
                      KT=p.KT, dt=p.dt, tol=p.tol, max_iter=p.max_iter, precision=prec,
                      j0_model=j0)
    m.set_state(st.Y, st.q, st.Yprev, st.u, st.lam if lay.n_lam else None)
    if ext is not None:
        m.set_external(ext.Fext, ext.Text, ext.follower)
    m.set_tether(teth.mask, teth.Y1, teth.u1)
    return m


def _system(segs, seed, history=False, dt=0.1, tol=1e-10):
    """Random filaments; the first and the last tethered with a moving base
    (Y_1 displaced, u_1 a small rotation)."""
    rng = np.random.default_rng(seed)
    lay = fo.Layout(segs)
    M = len(segs)
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=dt, tol=tol, max_iter=80)
    base = rng.uniform(0, 15.0 * M ** (1 / 3), size=(M, 3))
    t, mu = random_frames(rng, M)
    xi = 0.05 * rng.standard_normal((lay.S, 3))
    st = fo.initial_state(lay, p, base, t, mu, xi)
    if history:
        st.Yprev = st.Y + 0.01 * rng.standard_normal(st.Y.shape)
        st.u = 0.02 * rng.standard_normal((lay.S, 3))
    st.lam = 0.1 * rng.standard_normal((lay.n_lam, 3))
    mask = np.zeros(M, dtype=bool)
    mask[0] = mask[-1] = True
    Y1 = np.array([st.Y[lay.off_seg[i]] for i in range(M)]) + 0.05 * rng.standard_normal((M, 3))
    u1 = 0.03 * rng.standard_normal((M, 3))
    teth = fo.Tether(mask=mask, Y1=Y1, u1=u1)
    ext = fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1)),
                      Text=0.05 * rng.standard_normal((lay.S, 3)))
    return lay, p, st, ext, teth, rng


SEGS = [[20], [12, 5, 33], [16] * 5, [1, 7, 2]]


@pytest.mark.parametrize("segs", SEGS)
@pytest.mark.parametrize("history", [False, True])
def test_residual_parity(fil, segs, history):
    lay, p, st, ext, teth, rng = _system(segs, 3 + len(segs), history)
    Y1 = np.array([st.Y[lay.off_seg[i]] for i in range(lay.M)])
    Y1[teth.mask] = rng.standard_normal((int(teth.mask.sum()), 3))        # lambda_1
    u = 0.05 * rng.standard_normal((lay.S, 3))
    X = lay.join_X(Y1, u, rng.standard_normal((lay.n_lam, 3)))
    ref = fo.residual(lay, p, st, ext, X, tether=teth)
    with _gpu(fil, lay, p, st, ext, teth) as m:
        f = np.zeros(6 * lay.S)
        finf = m.residual(X, f)
        scale = max(1.0, np.abs(st.Y).max())
        np.testing.assert_allclose(f, ref, rtol=0, atol=1e-12 * scale)
        assert finf == np.abs(f).max()
        m.set_tether(None)                            # untied: the free residual
        m.residual(X, f)
        np.testing.assert_allclose(f, fo.residual(lay, p, st, ext, X), rtol=0,
                                   atol=1e-12 * scale)


@pytest.mark.parametrize("segs", [[20], [12, 5, 33], [16] * 5])
@pytest.mark.parametrize("history", [False, True])
@pytest.mark.parametrize("model", J0_MODELS)
def test_j0_solve_parity(fil, segs, history, model):
    lay, p, st, ext, teth, rng = _system(segs, 20 + len(segs), history)
    X0 = fo.initial_guess(lay, st, teth)
    ref_solver = fo.J0Solver(lay, fo.jacobian0_tethered(lay, p, st, X0, teth, model[1]))
    b = rng.standard_normal(6 * lay.S)
    ref = ref_solver.solve(b)
    with _gpu(fil, lay, p, st, ext, teth, j0=model[0]) as m:
        m.broyden_begin()
        Xg = np.zeros(6 * lay.S)
        m.get_iterate(Xg, None)
        np.testing.assert_allclose(Xg, X0, rtol=0, atol=1e-14 * max(1.0, np.abs(X0).max()))
        x = np.zeros(6 * lay.S)
        m.j0_solve(b, x)
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("model", J0_MODELS)
def test_broyden_iterates_match_oracle(fil, model):
    lay, p, st, ext, teth, _ = _system([16, 9, 20], 40, history=True, tol=1e-13)
    br = fo.begin_step(lay, p, st, ext, j0_model=model[1], tether=teth)
    with _gpu(fil, lay, p, st, ext, teth, j0=model[0]) as m:
        f0 = m.broyden_begin()
        assert abs(f0 - np.abs(br.f).max()) <= 1e-12 * max(1, np.abs(st.Y).max())
        X = np.zeros(6 * lay.S)
        f = np.zeros(6 * lay.S)
        for k in range(6):
            conv, _ = m.broyden_step()
            br.iterate()
            m.get_iterate(X, f)
            np.testing.assert_allclose(X, br.X, rtol=0, atol=1e-10 * np.abs(br.X).max())
            np.testing.assert_allclose(f, br.f, rtol=0, atol=1e-10 * max(1, np.abs(br.f).max()))
            if conv:
                break


def _motor(N=20, w=0.05, Sp=30.0):
    """The set-up of Sec. 5.2.1 (delta_0 = 4.5977a, 15 degrees to the motor
    axis e_z) at a Sperm number where the filament bends."""
    a, dL = 1.0, 2.2
    L = N * dL
    zeta = 4.0 * math.pi / (math.log(L / a) + 0.5)
    KB = zeta * w * L ** 4 / Sp
    dt = 2.0 * math.pi / w / 100.0
    lay = fo.Layout([N])
    p = fo.Params(a=a, eta=1.0, dL=dL, KB=KB, KT=KB, dt=dt, tol=1e-10, max_iter=100)
    th = math.radians(15.0)
    delta0 = 4.5977 * a
    st = fo.initial_state(lay, p, np.array([[delta0, 0.0, 0.0]]),
                          np.array([[math.sin(th), 0.0, math.cos(th)]]),
                          np.array([[0.0, 1.0, 0.0]]))

    def tether(j):
        ph = j * w * dt
        return fo.Tether(mask=np.array([True]),
                         Y1=np.array([[delta0 * math.cos(ph), delta0 * math.sin(ph), 0.0]]),
                         u1=np.array([[0.0, 0.0, w * dt]]))
    return lay, p, st, tether


@pytest.mark.parametrize("model", J0_MODELS)
def test_tether_set_once_keeps_j0_and_the_trajectory(fil, model):
    """A tether prescription set once (two filaments clamped where their first
    segments are: Y_1 held, u_1 = 0) lets J0 be kept (fil_set_j0_reuse) and
    the Broyden pairs be carried (fil_set_broyden_memory): every step stays on
    the oracle's trajectory (J0 built and memory reset every step) to the
    accuracy the tolerance gives, and setting the tether again makes the next
    step build J0."""
    lay, p, st, ext, teth, _ = _system([16, 9, 20], 41, tol=1e-10, dt=0.1)
    first = [lay.off_seg[i] for i in range(lay.M)]
    teth = fo.Tether(mask=teth.mask, Y1=np.array([st.Y[k] for k in first]),
                     u1=np.zeros((lay.M, 3)))
    with _gpu(fil, lay, p, st, ext, teth, j0=model[0]) as m:
        m.set_j0_reuse(5)
        m.set_broyden_memory(8)
        Y = np.zeros((lay.S, 3))
        for _ in range(8):
            st, _ = fo.step(lay, p, st, ext, j0_model=model[1], tether=teth)
            m.step()
            m.get_state(Y, None, None, None, None)
            np.testing.assert_allclose(Y, st.Y, rtol=0, atol=1e-8)
        builds, reuses = m.j0_stats()
        assert reuses >= 3, (builds, reuses)
        m.set_tether(teth.mask, teth.Y1, teth.u1)
        m.step()
        assert m.j0_stats()[0] == builds + 1


@pytest.mark.parametrize("model", J0_MODELS)
def test_motor_steps_match_oracle(fil, model):
    """Motor steps against the oracle; J0 reuse is requested and must not apply
    (the prescription is set anew for every step, and the tethered J0 columns
    follow it)."""
    lay, p, st, tether = _motor()
    with _gpu(fil, lay, p, st, None, tether(1), j0=model[0]) as m:
        m.set_j0_reuse(5)
        Y = np.zeros((lay.S, 3))
        lam = np.zeros((1, 6))
        for j in range(1, 13):
            teth = tether(j)
            m.set_tether(teth.mask, teth.Y1, teth.u1)
            st, it_ref = fo.step(lay, p, st, None, j0_model=model[1], tether=teth)
            it = m.step()
            m.get_state(Y, None, None, None, None)
            m.get_tether(lam)
            assert abs(it - it_ref) <= 1, (j, it, it_ref)
            np.testing.assert_allclose(Y, st.Y, rtol=0, atol=1e-8)
            np.testing.assert_allclose(Y[0], teth.Y1[0], rtol=0, atol=1e-12)
            np.testing.assert_allclose(lam, st.tlam, rtol=0, atol=1e-7 * np.abs(st.tlam).max())
        assert m.j0_stats()[1] == 0


@pytest.mark.parametrize("graph", [False, True])
def test_ensemble_with_tethers_matches_each_system(fil, graph):
    systems = [[14, 6], [20], [9, 9, 9]]
    lays, states, exts, teths = [], [], [], []
    p = None
    for k, segs in enumerate(systems):
        lay, p, st, ext, teth, _ = _system(segs, 60 + k, history=False, dt=0.2, tol=1e-10)
        st.lam = None
        lays.append(lay)
        states.append(st)
        exts.append(fo.External(Fext=ext.Fext))
        teths.append(teth)
    segs_all = [n for segs in systems for n in segs]
    with fil.Filaments(segs_all, fil_per_sys=[len(s) for s in systems], a=p.a, eta=p.eta,
                       dL=p.dL, KB=p.KB, KT=p.KT, dt=p.dt, tol=p.tol, max_iter=p.max_iter,
                       j0_model=1) as m:
        m.set_state(np.concatenate([s.Y for s in states]), np.concatenate([s.q for s in states]))
        m.set_external(np.concatenate([e.Fext for e in exts]), None, None)
        m.set_tether(np.concatenate([t.mask for t in teths]),
                     np.concatenate([t.Y1 for t in teths]), np.concatenate([t.u1 for t in teths]))
        m.set_graph(graph)
        Y = np.zeros((m.S, 3))
        for step in range(3):
            m.step()
            its, _ = m.sys_stats()
            m.get_state(Y, None, None, None, None)
            off = 0
            for k, lay in enumerate(lays):
                states[k], it_ref = fo.step(lay, p, states[k], exts[k], j0_model="rpy",
                                            tether=teths[k])
                assert abs(int(its[k]) - it_ref) <= 1, (step, k, its, it_ref)
                np.testing.assert_allclose(Y[off:off + lay.S], states[k].Y, rtol=0, atol=1e-8)
                off += lay.S


@pytest.mark.parametrize("model", J0_MODELS)
def test_clamped_elastica_on_gpu(fil, model):
    """The clamped filament under a tip force of fixed direction relaxes on the
    GPU to the elastica of Sec. 4.1 within the discretisation error, and to
    the oracle's discrete equilibrium far more closely."""
    N, ell, KB = 21, 44.0, 1.0
    dL = ell / (N - 1)
    F = 1.93 * KB / ell ** 2
    a = dL / 2.2
    tau = 6.0 * math.pi * a / dL * ell ** 4 / (12.4 * KB)
    p = fo.Params(a=a, eta=1.0, dL=dL, KB=KB, KT=KB, dt=0.5 * tau, tol=1e-10, max_iter=200)
    lay = fo.Layout([N])
    st = fo.initial_state(lay, p, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]),
                          np.array([[0.0, 1.0, 0.0]]))
    Fext = np.zeros((N, 3))
    Fext[-1] = [0.0, 0.0, -F]
    ext = fo.External(Fext=Fext)
    teth = fo.Tether(mask=np.array([True]), Y1=np.zeros((1, 3)), u1=np.zeros((1, 3)))
    ref = st
    for _ in range(40):
        ref, _ = fo.step(lay, p, ref, ext, j0_model=model[1], tether=teth)
    with _gpu(fil, lay, p, st, ext, teth, j0=model[0]) as m:
        for _ in range(40):
            m.step()
        q = np.zeros((N, 4))
        Y = np.zeros((N, 3))
        m.get_state(Y, q, None, None, None)
        lam = np.zeros((1, 6))
        m.get_tether(lam)
    t = fo.frames(q)[0]
    th = np.arccos(np.clip(-t[:, 2], -1.0, 1.0))
    th_ex = elastica.angles(dL * np.arange(N), ell, F, KB)
    E2 = math.sqrt(dL * np.sum((th - th_ex) ** 2))
    assert E2 < 4e-4
    th_ref = np.arccos(np.clip(-fo.frames(ref.q)[0][:, 2], -1.0, 1.0))
    np.testing.assert_allclose(th, th_ref, rtol=0, atol=1e-7)
    np.testing.assert_allclose(lam[0, :3], [0.0, 0.0, F], rtol=0, atol=1e-9)   # holds the load


def test_set_tether_states(fil):
    lay, p, st, ext, teth, _ = _system([8, 8], 1)
    with _gpu(fil, lay, p, st, ext, teth) as m:
        m.broyden_begin()
        with pytest.raises(fil.FilError, match="FIL_ESTATE"):
            m.set_tether(teth.mask, teth.Y1, teth.u1)
    with _gpu(fil, lay, p, st, ext, teth) as m:
        with pytest.raises(fil.FilError, match="FIL_EINVAL"):
            m.set_tether(teth.mask, None, None)
        lam = np.ones((lay.M, 6))
        m.get_tether(lam)
        np.testing.assert_array_equal(lam, 0.0)      # no tethered step yet
