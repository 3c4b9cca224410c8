"""GPU checks of the learned warm start inside the step (fil_warm_*): the
network inputs, the training targets and the prediction assembly against
the FP64 reference in oracle/warm.py, the selection rule (the start with the
smaller residual; a zero network reproduces the plain solve exactly), and
the gain of the trained network on the suspension workload."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filament as fo  # noqa: E402
from oracle import warm as ow  # noqa: E402
from paper_1903_12609_gb300.inputs import random_frames  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


def _system(segs, seed, tol=1e-11):
    rng = np.random.default_rng(seed)
    lay = fo.Layout(segs)
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.1, tol=tol, max_iter=60)
    M = len(segs)
    base = rng.uniform(0, 60.0, size=(M, 3))
    t, mu = random_frames(rng, M)
    xi = 0.05 * rng.standard_normal((lay.S, 3))
    st = fo.initial_state(lay, p, base, t, mu, xi)
    st.lam = 0.1 * rng.standard_normal((lay.n_lam, 3))
    ext = fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1)),
                      follower=rng.uniform(0, 1, M))
    return lay, p, st, ext


def _gpu(fil, lay, p, st, ext):
    m = fil.Filaments(lay.N, a=p.a, eta=p.eta, dL=p.dL, KB=p.KB, KT=p.KT, dt=p.dt, tol=p.tol,
                      max_iter=p.max_iter, precision=0, j0_model=1)
    m.set_state(st.Y, st.q, st.Yprev, st.u, st.lam)
    m.set_external(ext.Fext, ext.Text, ext.follower)
    return m


SEGS = [32, 20, 32, 32]


def test_features_match_reference(fil):
    lay, p, st, ext = _system(SEGS, 1)
    with _gpu(fil, lay, p, st, ext) as m:
        f = torch.zeros((lay.M, fil.MLP_IN), dtype=torch.float32, device="cuda")
        m.warm_features(f)
    ref = ow.features(lay, p, st, ext)
    np.testing.assert_allclose(f.cpu().numpy(), ref, rtol=2e-6, atol=2e-6 * np.abs(ref).max())
    assert np.all(f.cpu().numpy()[1] == 0)           # the 20-segment filament


def test_features_after_a_step_carry_its_correction(fil):
    lay, p, st, ext = _system(SEGS, 6)
    X_ex = fo.initial_guess(lay, st)
    br = fo.begin_step(lay, p, st, ext, j0_model="rpy")
    while not br.converged():
        br.iterate()
    st1 = fo.commit_step(lay, p, st, br.X)
    with _gpu(fil, lay, p, st, ext) as m:
        m.step()
        f = torch.zeros((lay.M, fil.MLP_IN), dtype=torch.float32, device="cuda")
        m.warm_features(f)
    ref = ow.features(lay, p, st1, ext, prev_corr=br.X - X_ex)
    f = f.cpu().numpy()
    np.testing.assert_allclose(f, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
    assert np.abs(f[:, -6 * 32:]).max() > 0


def test_targets_match_reference(fil):
    lay, p, st, ext = _system(SEGS, 2)
    X_ex = fo.initial_guess(lay, st)
    br = fo.begin_step(lay, p, st, ext, j0_model="rpy")
    while not br.converged():
        br.iterate()
    with _gpu(fil, lay, p, st, ext) as m:
        m.step()
        tg = torch.zeros((lay.M, fil.MLP_OUT), dtype=torch.float32, device="cuda")
        m.warm_targets(tg)
    ref = ow.targets(lay, st, br.X, X_ex)
    sc = np.abs(ref).max()
    np.testing.assert_allclose(tg.cpu().numpy(), ref, rtol=0, atol=1e-6 * sc + 1e-9)


def test_targets_need_a_committed_step(fil):
    lay, p, st, ext = _system(SEGS, 3)
    with _gpu(fil, lay, p, st, ext) as m:
        tg = torch.zeros((lay.M, fil.MLP_OUT), dtype=torch.float32, device="cuda")
        with pytest.raises(fil.FilError) as e:
            m.warm_targets(tg)
        assert e.value.status == fil.FIL_ESTATE


def _net(fil, bias_out=None, seed=0):
    net = fil.fil_mlp_create(64)
    prm = np.zeros(fil.MLP_NPARAM, dtype=np.float32)
    if bias_out is not None:
        prm[-fil.MLP_OUT:] = bias_out
    fil.fil_mlp_set_params(net, prm)
    return net


@pytest.mark.parametrize("mode", [0, 1])
def test_zero_network_reproduces_the_plain_solve(fil, mode):
    lay, p, st, ext = _system(SEGS, 4, tol=1e-9)
    Y = {}
    for use in (False, True):
        net = _net(fil)
        with _gpu(fil, lay, p, st, ext) as m:
            if use:
                fil.fil_warm_attach(m.ctx, net, mode)
            its = [m.step() for _ in range(3)]  # noqa: F841
            Y[use] = np.zeros((lay.S, 3))
            m.get_state(Y[use], None, None, None, None)
            stats = fil.fil_warm_stats(m.ctx)
            fil.fil_warm_attach(m.ctx, None)
        fil.fil_mlp_destroy(net)
        if use:   # ties keep the extrapolation; prediction-first takes the (equal) prediction
            assert stats == ((0, 3, 0) if mode == 0 else (3, 0, 0))
    np.testing.assert_array_equal(Y[True], Y[False])


def test_prediction_is_assembled_and_compared(fil):
    """A network whose output is a constant correction: X_pred = X_ex + R1 y,
    f(X_pred) as the oracle evaluates it, and the start with the smaller
    ||f||_inf is kept."""
    lay, p, st, ext = _system(SEGS, 5, tol=1e-9)
    y = (1e-3 * np.random.default_rng(0).standard_normal(fil.MLP_OUT)).astype(np.float32)
    net = _net(fil, bias_out=y)
    with _gpu(fil, lay, p, st, ext) as m:
        fil.fil_warm_attach(m.ctx, net)
        f0 = m.broyden_begin()
        X0 = np.zeros(6 * lay.S)
        m.get_iterate(X0, None)
        stats = fil.fil_warm_stats(m.ctx)
        fil.fil_warm_attach(m.ctx, None)
    fil.fil_mlp_destroy(net)
    X_ex = fo.initial_guess(lay, st)
    X_pred = ow.predict(lay, st, X_ex, np.tile(y.astype(np.float64), (lay.M, 1)))
    f_ex = np.abs(fo.residual(lay, p, st, ext, X_ex)).max()
    f_pred = np.abs(fo.residual(lay, p, st, ext, X_pred)).max()
    want = X_pred if f_pred < f_ex else X_ex
    assert stats[:2] == ((1, 0) if f_pred < f_ex else (0, 1))
    np.testing.assert_allclose(X0, want, rtol=0, atol=1e-9 * np.abs(want).max())
    assert abs(f0 - min(f_pred, f_ex)) <= 1e-9 * max(1.0, f0)


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1903_12609_gb300", "weights", "warmstart_n32.npz")


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained warm-start network")
def test_trained_network_starts_closer(fil):
    """What the trained network gains: the committed network on the full
    suspension workload (1000 filaments x 32, a seed it was not trained on),
    30 steps continuing from the same state as the plain solve. The start it
    gives has a smaller residual on average (mean log10 ||f(X_0)||_inf at least
    0.3 lower) than the extrapolation it was trained to correct (the order stored
    with the weights), the prediction is taken in most steps, and the Broyden
    iterations per step fall by at least 5%; every step converges to the same
    tolerance (the plain solve judges each step)."""
    from paper_1903_12609_gb300 import warmstart
    net = warmstart.load(WEIGHTS, max_batch=1024)
    ev = warmstart.evaluate(torch, net, 1000, 30, seed=11, order=warmstart.trained_order(WEIGHTS))
    fil.fil_mlp_destroy(net)
    plain, best, first = ev["plain"], ev["best_of_two"], ev["prediction_first"]
    assert best["log10_f0"] < plain["log10_f0"] - 0.3, ev
    assert best["from_prediction"] > best["from_extrapolation"], ev
    assert first["iters_per_step"] <= 0.95 * plain["iters_per_step"], ev
    assert best["iters_per_step"] <= 0.95 * plain["iters_per_step"], ev
