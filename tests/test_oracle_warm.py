"""Pins of the warm-start reference (oracle/warm.py): the network sees each
filament in its own frame, so its inputs and targets are invariant under a
rigid motion of the whole suspension; prediction inverts the targets; a
straight filament at rest has the closed-form frame coordinates."""
import numpy as np

from oracle import filament as fo
from oracle import warm as ow
from paper_1903_12609_gb300.inputs import random_frames


def _state(seed, segs=(32, 20, 32)):
    rng = np.random.default_rng(seed)
    lay = fo.Layout(list(segs))
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.1, tol=1e-10, max_iter=60)
    base = rng.uniform(0, 40.0, size=(lay.M, 3))
    t, mu = random_frames(rng, lay.M)
    st = fo.initial_state(lay, p, base, t, mu, 0.05 * rng.standard_normal((lay.S, 3)))
    st.lam = 0.1 * rng.standard_normal((lay.n_lam, 3))
    st.Yprev = st.Y + 0.01 * rng.standard_normal(st.Y.shape)
    st.u = 0.02 * rng.standard_normal((lay.S, 3))
    ext = fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1)), follower=rng.uniform(0, 1, lay.M))
    return lay, p, st, ext


def _rotate(lay, st, ext, q0, shift):
    R0 = fo.rotation_matrix(q0[None, :])[0]
    st2 = fo.State(Y=st.Y @ R0.T + shift, q=np.array([fo.qmul(q0, q) for q in st.q]),
                   Yprev=st.Yprev @ R0.T + shift, u=st.u @ R0.T, lam=st.lam @ R0.T,
                   steps=st.steps)
    ext2 = fo.External(Fext=ext.Fext @ R0.T, follower=ext.follower)
    return st2, ext2


def test_inputs_and_targets_are_invariant_under_rigid_motion():
    lay, p, st, ext = _state(1)
    q0 = np.array([0.3, -0.5, 0.7, 0.4])
    q0 /= np.linalg.norm(q0)
    st2, ext2 = _rotate(lay, st, ext, q0, np.array([5.0, -3.0, 11.0]))
    f1 = ow.features(lay, p, st, ext)
    f2 = ow.features(lay, p, st2, ext2)
    # quaternion components q_1^* q_n are invariant only up to the shared sign
    np.testing.assert_allclose(f2, f1, rtol=0, atol=1e-10 * np.abs(f1).max())
    rng = np.random.default_rng(2)
    X_ex = fo.initial_guess(lay, st)
    X_star = X_ex + 1e-3 * rng.standard_normal(X_ex.shape)
    R0 = fo.rotation_matrix(q0[None, :])[0]

    def rot_X(X, shift):
        out = (X.reshape(-1, 3) @ R0.T).ravel()
        for i in range(lay.M):
            out[6 * lay.off_seg[i]:6 * lay.off_seg[i] + 3] += shift
        return out
    sh = np.array([5.0, -3.0, 11.0])
    t1 = ow.targets(lay, st, X_star, X_ex)
    t2 = ow.targets(lay, st2, rot_X(X_star, sh), rot_X(X_ex, sh))
    np.testing.assert_allclose(t2, t1, rtol=0, atol=1e-12)


def test_prediction_inverts_the_targets():
    lay, p, st, ext = _state(3)
    X_ex = fo.initial_guess(lay, st)
    X_star = X_ex + 1e-2 * np.random.default_rng(4).standard_normal(X_ex.shape)
    y = ow.targets(lay, st, X_star, X_ex)
    Xp = ow.predict(lay, st, X_ex, y)
    for i, n in enumerate(lay.N):
        a, b = 6 * lay.off_seg[i], 6 * lay.off_seg[i + 1]
        want = X_star[a:b] if n == ow.SEG else X_ex[a:b]
        np.testing.assert_allclose(Xp[a:b], want, rtol=0, atol=1e-14)


def test_straight_filament_frame_coordinates():
    lay = fo.Layout([32])
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.1, tol=1e-10, max_iter=60)
    t = np.array([[0.0, 0.6, 0.8]])
    mu = np.array([[1.0, 0.0, 0.0]])
    st = fo.initial_state(lay, p, np.array([[1.0, 2.0, 3.0]]), t, mu)
    st.lam = np.zeros((lay.n_lam, 3))
    f = ow.features(lay, p, st, None)[0, :13 * 32].reshape(32, 13)
    np.testing.assert_allclose(f[:, 0], 2.2 * np.arange(32), atol=1e-12)
    np.testing.assert_allclose(f[:, 1:3], 0, atol=1e-12)
    np.testing.assert_allclose(np.abs(f[:, 3]), 1, atol=1e-12)
    np.testing.assert_allclose(f[:, 4:7], 0, atol=1e-12)
    np.testing.assert_allclose(f[:, 7:], 0, atol=1e-12)      # unloaded, unbent
