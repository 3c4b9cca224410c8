"""GPU parity of the steric barrier (Sec. 2.6; fil_set_steric) against the
oracle: residuals of dense configurations where many segment pairs sit within
the barrier's range 2 chi a, timesteps of filament bundles inside its range,
no barrier across the systems of an ensemble, and the overflow status of the
cell grid.

Tolerances are those of the FP64 residual and step parity tests (1e-12 of the
largest position for residual entries, 1e-8 absolute for positions after a
few steps at a Broyden tolerance of 1e-10).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filament as fo  # noqa: E402
from oracle import steric  # noqa: E402
from paper_1903_12609_gb300.inputs import random_frames  # noqa: E402

pytestmark = pytest.mark.gpu

CHI = 1.1


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


def _params(FS, **kw):
    base = dict(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.1, tol=1e-10, max_iter=80,
                FS=FS, chi=CHI)
    base.update(kw)
    return fo.Params(**base)


def _gpu(fil, lay, p, st, ext, fil_per_sys=None):
    m = fil.Filaments(lay.N, fil_per_sys=fil_per_sys, a=p.a, eta=p.eta, dL=p.dL, KB=p.KB,
                      KT=p.KT, dt=p.dt, tol=p.tol, max_iter=p.max_iter)
    m.set_state(st.Y, st.q, st.Yprev, st.u, st.lam if lay.n_lam else None)
    m.set_external(ext.Fext, ext.Text, ext.follower)
    m.set_steric(p.FS, p.chi)
    return m


def _cloud(segs, box, seed, p):
    """Filaments with random bases in a small cube: many crossings."""
    rng = np.random.default_rng(seed)
    lay = fo.Layout(segs)
    M = len(segs)
    base = rng.uniform(0, box, size=(M, 3))
    t, mu = random_frames(rng, M)
    xi = 0.05 * rng.standard_normal((lay.S, 3))
    st = fo.initial_state(lay, p, base, t, mu, xi)
    st.lam = 0.1 * rng.standard_normal((lay.n_lam, 3))
    ext = fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1)),
                      Text=0.05 * rng.standard_normal((lay.S, 3)))
    return lay, st, ext, rng


def _bundle(n_side, n_seg, gap, seed, p, tilt=0.3):
    """n_side x n_side parallel filaments on a square lattice of spacing gap
    (< 2 chi a: lattice neighbours are within the barrier's range)."""
    rng = np.random.default_rng(seed)
    d = np.array([np.sin(tilt), 0.0, np.cos(tilt)])
    e1 = np.array([0.0, 1.0, 0.0])
    e2 = np.cross(d, e1)
    base = np.array([i * gap * e1 + j * gap * e2 for i in range(n_side) for j in range(n_side)])
    M = n_side * n_side
    lay = fo.Layout([n_seg] * M)
    t = np.tile(d, (M, 1))
    mu = np.tile(e1, (M, 1))
    xi = 0.02 * rng.standard_normal((lay.S, 3))
    st = fo.initial_state(lay, p, base, t, mu, xi)
    ext = fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1)))
    return lay, st, ext


def _pairs_in_range(lay, Y, chi):
    fil_of = np.repeat(np.arange(lay.M), lay.N)
    n = 0
    for i in range(lay.S):
        r = np.linalg.norm(Y[i + 1:] - Y[i], axis=1)
        m = np.arange(i + 1, lay.S)
        neigh = (fil_of[m] == fil_of[i]) & (m == i + 1)
        n += int(np.sum((r < 2 * chi) & ~neigh))
    return n


@pytest.mark.parametrize("segs,box", [([12] * 8, 8.0), ([1, 5, 33, 20], 4.0), ([24] * 10, 9.0)])
def test_residual_parity_dense(fil, segs, box):
    p = _params(FS=0.7)
    lay, st, ext, rng = _cloud(segs, box, len(segs), p)
    Y1 = np.array([st.Y[lay.off_seg[i]] for i in range(lay.M)])
    X = lay.join_X(Y1, 0.02 * rng.standard_normal((lay.S, 3)),
                   rng.standard_normal((lay.n_lam, 3)))
    Yx = fo.unpack(lay, p, X, st.q)[2]
    assert _pairs_in_range(lay, Yx, CHI) >= 4
    ref = fo.residual(lay, p, st, ext, X, nthreads=4)
    ref0 = fo.residual(lay, _params(FS=0.0), st, ext, X, nthreads=4)
    assert np.abs(ref - ref0).max() > 1e-3          # the barrier changes the residual
    with _gpu(fil, lay, p, st, ext) as m:
        f = np.zeros(6 * lay.S)
        finf = m.residual(X, f)
        scale = max(1.0, np.abs(st.Y).max(), np.abs(ref).max())
        np.testing.assert_allclose(f, ref, rtol=0, atol=1e-12 * scale)
        assert finf == np.abs(f).max()
        m.set_steric(0.0, CHI)                      # switched off again
        m.residual(X, f)
        np.testing.assert_allclose(f, ref0, rtol=0, atol=1e-12 * scale)


def test_barrier_force_alone(fil):
    """No gravity: the residual is linear in the forces, so its difference to
    the barrier-free residual is the barrier's contribution alone (the
    mobility of F^B, scaled by the step); compared with the oracle's."""
    p = _params(FS=1.3)
    lay, st, ext, rng = _cloud([10] * 12, 7.0, 3, p)
    ext = fo.External(Fext=np.zeros((lay.S, 3)))
    X = fo.initial_guess(lay, st)
    Yx = fo.unpack(lay, p, X, st.q)[2]
    assert _pairs_in_range(lay, Yx, CHI) >= 10
    FB = steric.barrier_forces(lay.N, Yx, p.a, p.FS, p.chi)
    assert np.abs(FB).max() > 0
    ref = fo.residual(lay, p, st, ext, X) - fo.residual(lay, _params(FS=0.0), st, ext, X)
    with _gpu(fil, lay, p, st, ext) as m:
        f1 = np.zeros(6 * lay.S)
        f0 = np.zeros(6 * lay.S)
        m.residual(X, f1)
        m.set_steric(0.0, CHI)
        m.residual(X, f0)
    np.testing.assert_allclose(f1 - f0, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_bundle_steps_match_oracle(fil):
    """A 3 x 3 bundle at lattice spacing 2.1a (inside the range 2.2a) sediments
    for a few steps with the barrier active throughout."""
    p = _params(FS=1.0, dt=0.1)
    lay, st, ext = _bundle(3, 16, 2.1, 0, p)
    assert _pairs_in_range(lay, st.Y, CHI) >= 100
    with _gpu(fil, lay, p, st, ext) as m:
        Y = np.zeros((lay.S, 3))
        for step in range(4):
            st, it_ref = fo.step(lay, p, st, ext)
            it = m.step()
            m.get_state(Y, None, None, None, None)
            assert abs(it - it_ref) <= 1, (step, it, it_ref)
            np.testing.assert_allclose(Y, st.Y, rtol=0, atol=1e-8)
    assert _pairs_in_range(lay, st.Y, CHI) >= 100


@pytest.mark.parametrize("graph", [False, True])
def test_no_barrier_across_systems(fil, graph):
    """Two copies of one bundle at the same coordinates in one ensemble: were
    the barrier to act across systems, coincident segments would repel; each
    system must step exactly as the oracle's single bundle."""
    p = _params(FS=1.0, dt=0.1)
    lay, st, ext = _bundle(2, 12, 2.05, 1, p)
    lay2 = fo.Layout(lay.N * 2)
    st2 = fo.State(Y=np.concatenate([st.Y, st.Y]), q=np.concatenate([st.q, st.q]))
    ext2 = fo.External(Fext=np.concatenate([ext.Fext, ext.Fext]))
    with _gpu(fil, lay2, p, st2, ext2, fil_per_sys=[lay.M, lay.M]) as m:
        m.set_graph(graph)
        Y = np.zeros((lay2.S, 3))
        for step in range(3):
            st, it_ref = fo.step(lay, p, st, ext)
            m.step()
            its, _ = m.sys_stats()
            m.get_state(Y, None, None, None, None)
            for k in range(2):
                assert abs(int(its[k]) - it_ref) <= 1
                np.testing.assert_allclose(Y[k * lay.S:(k + 1) * lay.S], st.Y, rtol=0, atol=1e-8)


def test_overflow_status_and_recovery(fil):
    """60 single-segment filaments inside a unit cube: every segment has 59
    others within range (more than the 48 a segment keeps) -- FIL_EOVERFLOW,
    after which the context still works."""
    p = _params(FS=1.0)
    lay = fo.Layout([1] * 60)
    rng = np.random.default_rng(0)
    base = rng.uniform(0, 1.0, size=(60, 3))
    t, mu = random_frames(rng, 60)
    st = fo.initial_state(lay, p, base, t, mu, np.zeros((60, 3)))
    ext = fo.External(Fext=np.zeros((60, 3)))
    X = fo.initial_guess(lay, st)
    with _gpu(fil, lay, p, st, ext) as m:
        f = np.zeros(6 * lay.S)
        with pytest.raises(fil.FilError, match="FIL_EOVERFLOW"):
            m.residual(X, f)
        m.set_steric(0.0, CHI)
        m.residual(X, f)
        ref = fo.residual(lay, _params(FS=0.0), st, ext, X)
        np.testing.assert_allclose(f, ref, rtol=0, atol=1e-12)


def test_set_steric_rejects_bad_arguments(fil):
    p = _params(FS=0.0)
    lay, st, ext, _ = _cloud([8, 8], 20.0, 0, p)
    with _gpu(fil, lay, p, st, ext) as m:
        for FS, chi in [(-1.0, 1.1), (1.0, 1.0), (1.0, 0.5), (float("nan"), 1.1),
                        (1.0, float("inf"))]:
            with pytest.raises(fil.FilError, match="FIL_EINVAL"):
                m.set_steric(FS, chi)
