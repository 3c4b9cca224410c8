"""The seeded input recipe (shared by the oracle and the GPU tests, no method
arithmetic): the suspension and ensemble generators produce the shapes, box
size, frames, loads and parameters the workload description states."""
import numpy as np

from paper_1903_12609_gb300 import inputs


def test_suspension_recipe():
    wl, base, t, mu, Fext, follower = inputs.suspension(1000, 32, seed=0)
    S = 32000
    assert wl.seg_per_fil == [32] * 1000 and Fext.shape == (S, 3) and follower.shape == (1000,)
    # box of the 2% volume fraction: S (4/3) pi a^3 / side^3 = 0.02 -> side ~ 188.5 a
    side = inputs.box_side(S, 0.02, 1.0)
    assert abs(S * 4.0 / 3.0 * np.pi / side ** 3 - 0.02) < 1e-12
    assert abs(side - 188.5) < 0.1
    assert np.all(base >= 0.0) and np.all(base <= side)
    # orthonormal frames, tangents spread over the sphere
    np.testing.assert_allclose(np.linalg.norm(t, axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(mu, axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.sum(t * mu, axis=1), 0.0, atol=1e-12)
    assert np.all(np.abs(t.mean(axis=0)) < 0.1)
    # physics: B = L^3 W / K_B = 1000, dt = T / 200 with T = eta L / W, tol 1e-4
    L = 32 * wl.dL
    assert abs(L ** 3 * wl.W / wl.KB - 1000.0) < 1e-9
    assert abs(wl.dt - wl.eta * L / wl.W / 200.0) < 1e-12 and wl.tol == 1e-4
    # first half sediments (-W dL per segment, no follower), second half is driven
    # by a tip follower force with f L^2 / K_B = 100 and carries no weight
    Fz = Fext[:, 2].reshape(1000, 32)
    assert np.all(Fz[:500] == -wl.W * wl.dL) and np.all(Fz[500:] == 0.0)
    assert np.all(Fext[:, :2] == 0.0)
    assert np.all(follower[:500] == 0.0)
    np.testing.assert_allclose(follower[500:] * L ** 2 / wl.KB, 100.0, rtol=1e-12)


def test_suspension_has_no_overlapping_segments():
    wl, base, t, mu, _, _ = inputs.suspension(200, 32, seed=3, volume_fraction=0.05)
    Y = np.concatenate([base[i] + np.arange(32)[:, None] * wl.dL * t[i] for i in range(200)])
    fil = np.repeat(np.arange(200), 32)
    d2 = np.sum((Y[:, None, :] - Y[None, :, :]) ** 2, axis=2)
    other = fil[:, None] != fil[None, :]
    assert d2[other].min() >= 4.0 * wl.a ** 2


def test_generators_are_seeded():
    a = inputs.suspension(50, 32, seed=5)
    b = inputs.suspension(50, 32, seed=5)
    c = inputs.suspension(50, 32, seed=6)
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a[1], c[1])


def test_ensemble_recipe():
    wl, fps, segs, base, t, mu, Fext, follower = inputs.ensemble(16, seed=0)
    assert len(fps) == 16 and sum(fps) == len(segs) == base.shape[0] == follower.shape[0]
    assert all(1 <= f <= 64 for f in fps) and all(16 <= n <= 48 for n in segs)
    assert Fext.shape == (sum(segs), 3)
    # in every system the first half sediments and the rest is follower-driven
    off = 0
    seg_off = np.concatenate([[0], np.cumsum(segs)])
    for f in fps:
        passive = np.arange(f) < f // 2
        for j in range(f):
            i = off + j
            rows = slice(seg_off[i], seg_off[i + 1])
            L = segs[i] * wl.dL
            if passive[j]:
                assert follower[i] == 0.0 and np.all(Fext[rows, 2] == -wl.W * wl.dL)
            else:
                assert np.all(Fext[rows, 2] == 0.0)
                np.testing.assert_allclose(follower[i] * L ** 2 / wl.KB, 100.0, rtol=1e-12)
        off += f
