"""GPU parity of ensembles of independent systems (fil_create_ensemble): every
system of the batch behaves exactly as the oracle run on that system alone --
the mobility apply (no coupling across systems) and whole timesteps with
per-system Broyden convergence (a system that converges first keeps its
iterate while the others continue)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filament as fo  # noqa: E402
from oracle import rpy  # noqa: E402
from paper_1903_12609_gb300.inputs import random_frames  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


# systems: lists of segment counts (ragged, tiles and chunks cut mid-way)
SYSTEMS = [[16], [20, 33, 7], [48] * 6, [1, 2, 3], [32] * 9, [17, 40]]


def _positions(rng, segs, box):
    Y = []
    for n in segs:
        base = rng.uniform(0, box, 3)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y.append(base + 2.2 * np.arange(n)[:, None] * d)
    return np.concatenate(Y)


@pytest.mark.parametrize("tune", [False, True, (128, 1, 3), (128, 1, 2, 2)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_mobility_is_block_diagonal_over_systems(fil, prec, tune):
    """The ensemble apply couples only segments of the same system, under the
    default schedule, the autotuner's choice and schedules set by hand (the
    last with the source split, which the FP64 path does not have)."""
    if isinstance(tune, tuple) and len(tune) > 3 and prec == 0:
        pytest.skip("no source split on the FP64 path")
    rng = np.random.default_rng(prec)
    Ys, FTs = [], []
    for segs in SYSTEMS:
        Ys.append(_positions(rng, segs, 30.0))      # systems overlap in space
        FTs.append(rng.standard_normal((sum(segs), 6)))
    Y, FT = np.concatenate(Ys), np.concatenate(FTs)
    segs_all = [n for segs in SYSTEMS for n in segs]
    with fil.Filaments(segs_all, fil_per_sys=[len(s) for s in SYSTEMS], precision=prec,
                       max_iter=10) as m:
        if isinstance(tune, tuple):
            m.set_pair_schedule(*tune[:3])
            if len(tune) > 3:
                m.set_source_split(tune[3])
        elif tune:
            m.set_state(Y, np.tile([1.0, 0.0, 0.0, 0.0], (len(Y), 1)))
            tile, ctas, ms = m.autotune(2)
            assert tile in (128, 256) and ctas >= 1 and ms > 0
            assert m.pair_schedule()[0] == tile
        VW = np.zeros_like(FT)
        m.mobility_apply(Y, FT, VW)
    off = 0
    for Yi, FTi in zip(Ys, FTs):
        ref, ref_abs = rpy.apply(Yi, FTi, with_abs=True)
        got = VW[off:off + len(Yi)]
        if prec == 0:
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        else:
            assert np.all(np.abs(got - ref) <= 144 * 2.0 ** -24 * ref_abs + 1e-300)
        off += len(Yi)


def _system(segs, seed):
    rng = np.random.default_rng(seed)
    lay = fo.Layout(segs)
    M = len(segs)
    base = rng.uniform(0, 20.0 * M ** (1 / 3), size=(M, 3))
    t, mu = random_frames(rng, M)
    xi = 0.05 * rng.standard_normal((lay.S, 3))
    return lay, base, t, mu, xi, rng


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("j0", [(0, "drag"), (1, "rpy")])
def test_ensemble_steps_match_each_system_alone(fil, j0, graph):
    systems = [[16], [20, 33, 7], [30] * 5, [1, 2, 3]]
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.2, tol=1e-10, max_iter=80)
    states, exts, lays = [], [], []
    for i, segs in enumerate(systems):
        lay, base, t, mu, xi, rng = _system(segs, 10 + i)
        st = fo.initial_state(lay, p, base, t, mu, xi)
        ext = fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1)),
                          follower=rng.uniform(0, 2, lay.M))
        states.append(st)
        exts.append(ext)
        lays.append(lay)
    segs_all = [n for segs in systems for n in segs]
    with fil.Filaments(segs_all, fil_per_sys=[len(s) for s in systems], a=p.a, eta=p.eta,
                       dL=p.dL, KB=p.KB, KT=p.KT, dt=p.dt, tol=p.tol, max_iter=p.max_iter,
                       j0_model=j0[0]) as m:
        m.set_state(np.concatenate([s.Y for s in states]), np.concatenate([s.q for s in states]))
        m.set_external(np.concatenate([e.Fext for e in exts]), None,
                       np.concatenate([e.follower for e in exts]))
        m.set_graph(graph)
        S = m.S
        Y = np.zeros((S, 3))
        for step in range(3):
            it_all = m.step()
            its, finf = m.sys_stats()
            m.get_state(Y, None, None, None, None)
            off = 0
            for k, lay in enumerate(lays):
                states[k], it_ref = fo.step(lay, p, states[k], exts[k], j0_model=j0[1])
                assert abs(int(its[k]) - it_ref) <= 1, (step, k, its, it_ref)
                np.testing.assert_allclose(Y[off:off + lay.S], states[k].Y, rtol=0, atol=1e-8)
                assert finf[k] <= p.tol * p.a
                off += lay.S
            assert it_all == its.max()


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_iterations_reproduce_launched_iterations(fil, prec):
    """A single system stepped with and without the graph-captured Broyden
    iteration: bit-identical trajectories and iteration counts."""
    lay, base, t, mu, xi, rng = _system([20, 30, 12], 5)
    # FP32 pair sums bound the attainable residual: a looser tolerance for them
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.2,
                  tol=1e-9 if prec == 0 else 1e-6, max_iter=60)
    st = fo.initial_state(lay, p, base, t, mu, xi)
    Fext = np.tile([0.0, 0.0, -2.2], (lay.S, 1))
    out = {}
    for graph in (False, True):
        with fil.Filaments(lay.N, a=p.a, eta=p.eta, dL=p.dL, KB=p.KB, KT=p.KT, dt=p.dt,
                           tol=p.tol, max_iter=p.max_iter, precision=prec, j0_model=1) as m:
            m.set_state(st.Y, st.q)
            m.set_external(Fext, None, None)
            m.set_graph(graph)
            its = [m.step() for _ in range(4)]
            Y = np.zeros((lay.S, 3))
            m.get_state(Y, None, None, None, None)
            out[graph] = (its, Y)
    assert out[True][0] == out[False][0]
    np.testing.assert_array_equal(out[True][1], out[False][1])


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("j0", [(0, "drag"), (1, "rpy")])
@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_ensemble_converges_close_to_fp64(fil, j0, prec, split):
    """The mixed modes (FP32 pair sums; FIL_MIXED also FP32 J0 solves and FP32
    Broyden history) on an ensemble: every system converges to the oracle's FP64
    trajectory within the accuracy its tolerance allows, and every system's
    ||f||_inf meets it; with the one-target pair kernel, unsplit and with its
    sources split over two halves of each CTA (late iterations then run the
    split kernel over the short list of tiles still active)."""
    systems = [[16], [20, 33, 7], [30] * 5, [1, 2, 3]]
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.2, tol=1e-6, max_iter=80)
    states, exts, lays = [], [], []
    for i, segs in enumerate(systems):
        lay, base, t, mu, xi, rng = _system(segs, 30 + i)
        states.append(fo.initial_state(lay, p, base, t, mu, xi))
        exts.append(fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1))))
        lays.append(lay)
    segs_all = [n for segs in systems for n in segs]
    with fil.Filaments(segs_all, fil_per_sys=[len(s) for s in systems], a=p.a, eta=p.eta,
                       dL=p.dL, KB=p.KB, KT=p.KT, dt=p.dt, tol=p.tol, max_iter=p.max_iter,
                       precision=prec, j0_model=j0[0]) as m:
        m.set_state(np.concatenate([s.Y for s in states]), np.concatenate([s.q for s in states]))
        m.set_external(np.concatenate([e.Fext for e in exts]), None, None)
        m.set_pair_schedule(128, 1, 2)
        m.set_source_split(split)
        Y = np.zeros((m.S, 3))
        for _ in range(3):
            m.step()
            _, finf = m.sys_stats()
            assert np.all(finf <= p.tol * p.a)
            for k, lay in enumerate(lays):
                states[k], _ = fo.step(lay, p, states[k], exts[k], j0_model=j0[1])
        m.get_state(Y, None, None, None, None)
    off = 0
    for k, lay in enumerate(lays):
        np.testing.assert_allclose(Y[off:off + lay.S], states[k].Y, rtol=0, atol=1e-4)
        off += lay.S


@pytest.mark.parametrize("carry", [0, 8])
@pytest.mark.parametrize("j0", [(0, "drag"), (1, "rpy")])
def test_ensemble_with_j0_reuse_stays_on_each_systems_trajectory(fil, j0, carry):
    """An ensemble stepped with J0 kept for up to 3 steps (fil_set_j0_reuse),
    and with 8 Broyden pairs carried while it is kept (fil_set_broyden_memory;
    systems converge at different iterations, so later pairs hold zero rows
    for the early ones): every system meets the tolerance at every step and
    stays on the oracle's trajectory of that system alone (J0 built and the
    memory reset every step) to the accuracy the tolerance gives."""
    systems = [[16], [20, 33, 7], [30] * 5, [1, 2, 3]]
    p = fo.Params(a=1.0, eta=1.0, dL=2.2, KB=2.0, KT=1.5, dt=0.2, tol=1e-10, max_iter=80)
    states, exts, lays = [], [], []
    for i, segs in enumerate(systems):
        lay, base, t, mu, xi, rng = _system(segs, 40 + i)
        states.append(fo.initial_state(lay, p, base, t, mu, xi))
        exts.append(fo.External(Fext=np.tile([0.0, 0.0, -2.2], (lay.S, 1))))
        lays.append(lay)
    segs_all = [n for segs in systems for n in segs]
    with fil.Filaments(segs_all, fil_per_sys=[len(s) for s in systems], a=p.a, eta=p.eta,
                       dL=p.dL, KB=p.KB, KT=p.KT, dt=p.dt, tol=p.tol, max_iter=p.max_iter,
                       j0_model=j0[0]) as m:
        m.set_state(np.concatenate([s.Y for s in states]), np.concatenate([s.q for s in states]))
        m.set_external(np.concatenate([e.Fext for e in exts]), None, None)
        m.set_j0_reuse(3)
        m.set_broyden_memory(carry)
        Y = np.zeros((m.S, 3))
        for step in range(7):
            m.step()
            _, finf = m.sys_stats()
            assert np.all(finf <= p.tol * p.a)
            m.get_state(Y, None, None, None, None)
            off = 0
            for k, lay in enumerate(lays):
                states[k], _ = fo.step(lay, p, states[k], exts[k], j0_model=j0[1])
                np.testing.assert_allclose(Y[off:off + lay.S], states[k].Y, rtol=0, atol=1e-8)
                off += lay.S
        assert m.j0_stats()[1] >= 2
