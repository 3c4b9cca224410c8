"""GPU parity of the RPY mobility apply (fil_mobility_apply) against the oracle.

FP64 path: normwise relative error <= 1e-12 per call.
Mixed paths (FP32 pair sums; FIL_MIXED and FIL_PAIR32 run the same apply):
every component within
    |v_gpu - v_oracle| <= C_MIXED * 2^-24 * B
where B is the oracle's sum over pairs of |parts of M_nm| (|F|, |T|) for that
component. C_MIXED = 4 * 32 + 16: each group of 32 sources is accumulated by
4 FP32 FMAs per component and pair (<= 128 roundings of the running sum), each
pair term carries <= ~12 roundings (hi/lo difference, rsqrt, products) and the
inputs are rounded to FP32 once; the compensated fold of the group sums and
the float-float sums of the partials add O(u^2).
"""
import os

import numpy as np
import pytest

from conftest import MIXED_MAX_C

torch = pytest.importorskip("torch")

from oracle import rpy  # noqa: E402
from paper_1903_12609_gb300.inputs import mobility_inputs  # noqa: E402

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
C_MIXED = 4 * 32 + 16


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


def _gpu_apply(fil, segs, Y, FT, prec, host=False, a=1.0, eta=1.0):
    with fil.Filaments(segs, a=a, eta=eta, precision=prec) as m:
        if host:
            VW = np.zeros((Y.shape[0], 6))
            m.mobility_apply(np.ascontiguousarray(Y), np.ascontiguousarray(FT), VW)
            return VW
        Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
        FTd = torch.from_numpy(np.ascontiguousarray(FT)).cuda()
        VW = torch.empty((Y.shape[0], 6), dtype=torch.float64, device="cuda")
        m.mobility_apply(Yd, FTd, VW)
        torch.cuda.synchronize()
        return VW.cpu().numpy()


def _check_mixed(got, ref, ref_abs, name=None):
    bound = C_MIXED * U32 * ref_abs
    err = np.abs(got - ref)
    c = err / np.maximum(ref_abs, 1e-300) / U32
    if name is None:
        name = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    MIXED_MAX_C[name] = max(MIXED_MAX_C.get(name, 0.0), float(c.max()))
    assert np.all(err <= bound), "max c = %.2f" % float(c.max())
    # typical error is a few ulps of B
    assert np.median(c) < 8, "median c = %.2f" % float(np.median(c))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_c1_workload_parity(fil, prec):
    """100 random-walk filaments x 32 segments, 5% volume fraction, N(0,1) loads."""
    Y, FT = mobility_inputs(100, 32, seed=0)
    ref, ref_abs = rpy.apply(Y, FT, with_abs=True, nthreads=8)
    got = _gpu_apply(fil, [32] * 100, Y, FT, prec)
    if prec == fil.FIL_FP64:
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    else:
        _check_mixed(got, ref, ref_abs)


@pytest.mark.parametrize("segs", [[1], [7], [255], [1, 256], [3, 254, 2], [100] * 5 + [13],
                                  [64] * 17 + [5]])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_ragged_sizes(fil, segs, prec):
    S = sum(segs)
    rng = np.random.default_rng(S)
    Y = rng.uniform(0, max(4.0, S ** (1 / 3) * 3.0), size=(S, 3))
    FT = rng.standard_normal((S, 6))
    ref, ref_abs = rpy.apply(Y, FT, with_abs=True, nthreads=8)
    got = _gpu_apply(fil, segs, Y, FT, prec)
    if prec == fil.FIL_FP64:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    else:
        _check_mixed(got, ref, ref_abs)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_overlaps_and_coincident_segments(fil, prec):
    """Dense cluster: most pairs overlap (r < 2a); two pairs coincide exactly."""
    rng = np.random.default_rng(11)
    Y = rng.uniform(0, 3.0, size=(300, 3))
    Y[5] = Y[4]
    Y[77] = Y[200]
    FT = rng.standard_normal((300, 6))
    a, eta = 1.3, 0.8
    ref, ref_abs = rpy.apply(Y, FT, a, eta, with_abs=True)
    got = _gpu_apply(fil, [300], Y, FT, prec, a=a, eta=eta)
    if prec == fil.FIL_FP64:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    else:
        _check_mixed(got, ref, ref_abs)


@pytest.mark.parametrize("shift", [(150.0, -90.0, 200.0), (-3000.0, 2500.0, 1000.0)])
def test_far_from_origin(fil, shift):
    """The C1 workload moved away from the origin. The far-form loop forms d
    from the FP32 hi parts of the coordinates (their rounding kept for pairs
    beyond R_c = 4a; closer pairs are recomputed with hi/lo differences); the
    coordinates are taken relative to the first segment, so the error does not
    grow with the distance from the origin. Same bound as everywhere."""
    Y, FT = mobility_inputs(100, 32, seed=9)
    Y = Y + np.asarray(shift)
    ref, ref_abs = rpy.apply(Y, FT, with_abs=True, nthreads=8)
    got = _gpu_apply(fil, [32] * 100, Y, FT, fil.FIL_PAIR32)
    _check_mixed(got, ref, ref_abs)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_full_size_sampled_rows(fil, prec):
    """32 000 segments (the full-suspension size): sampled targets vs the oracle."""
    Y, FT = mobility_inputs(1000, 32, volume_fraction=0.02, seed=3)
    got = _gpu_apply(fil, [32] * 1000, Y, FT, prec)
    rows = np.concatenate([[0, 1, 255, 256, 31999], np.random.default_rng(4).integers(0, 32000, 59)])
    ref, ref_abs = rpy.apply_rows(Y, FT, rows, with_abs=True, nthreads=8)
    if prec == fil.FIL_FP64:
        np.testing.assert_allclose(got[rows], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    else:
        _check_mixed(got[rows], ref, ref_abs)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_deterministic_and_host_pointers(fil, prec):
    Y, FT = mobility_inputs(20, 32, seed=5)
    a = _gpu_apply(fil, [32] * 20, Y, FT, prec)
    b = _gpu_apply(fil, [32] * 20, Y, FT, prec)
    c = _gpu_apply(fil, [32] * 20, Y, FT, prec, host=True)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)


def test_zero_load_gives_zero(fil):
    Y, FT = mobility_inputs(4, 32, seed=6)
    got = _gpu_apply(fil, [32] * 4, Y, np.zeros_like(FT), 1)
    assert np.all(got == 0.0)


def test_apply_captured_in_a_cuda_graph(fil):
    """fil_mobility_apply with device arrays allocates nothing and does not
    synchronise, so it can be captured in a CUDA graph on the context's stream:
    replays give the launched result bit for bit, and the profiling events
    captured with it time the replayed pair kernels."""
    Y, FT = mobility_inputs(20, 32, seed=12)
    S = Y.shape[0]
    stream = torch.cuda.Stream()
    with fil.Filaments([32] * 20, precision=fil.FIL_PAIR32, stream=stream.cuda_stream) as m:
        Yd = torch.from_numpy(Y).cuda()
        FTd = torch.from_numpy(FT).cuda()
        ref = torch.empty((S, 6), dtype=torch.float64, device="cuda")
        m.mobility_apply(Yd, FTd, ref)
        torch.cuda.synchronize()
        out = torch.zeros((S, 6), dtype=torch.float64, device="cuda")
        m.profile(True)
        m.profile_read()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
            for _ in range(3):
                m.mobility_apply(Yd, FTd, out)
        out.zero_()
        torch.cuda.synchronize()
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        n, ms = m.profile_read()
        m.profile(False)
        assert n == 3 and ms > 0.0
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


SCHEDULES = [(256, 2, 4, 1), (128, 1, 4, 1), (128, 1, 1, 1), (256, 2, 1, 1), (128, 1, 2, 2),
             (128, 1, 1, 2)]


@pytest.mark.parametrize("sched", SCHEDULES)
@pytest.mark.parametrize("segs", [[32] * 100, [64] * 17 + [5], [3, 254, 2]])
def test_pair_schedules(fil, sched, segs):
    """Every pair schedule the autotuner chooses from (256-target tiles with 2
    targets per thread, 128-target tiles with 1 and the sources of a chunk
    split over one or two halves of the CTA, one to several resident CTAs per
    SM), set by hand, against the oracle."""
    S = sum(segs)
    rng = np.random.default_rng(S + sched[0] + sched[1])
    Y = rng.uniform(0, max(4.0, S ** (1 / 3) * 3.0), size=(S, 3))
    FT = rng.standard_normal((S, 6))
    ref, ref_abs = rpy.apply(Y, FT, with_abs=True, nthreads=8)
    with fil.Filaments(segs, precision=fil.FIL_PAIR32) as m:
        m.set_pair_schedule(*sched[:3])
        m.set_source_split(sched[3])
        assert m.pair_schedule() == sched[:3] and m.source_split() == sched[3]
        VW = np.zeros((S, 6))
        m.mobility_apply(Y, FT, VW)
    _check_mixed(VW, ref, ref_abs)


def test_source_split_on_the_c1_workload(fil):
    """The split kernel on the 3200-segment random-walk suspension (5% volume
    fraction: many close groups, own groups on every diagonal chunk) against the
    oracle, and against the unsplit kernel (the same pair terms, summed in
    another order: within the mixed bound of each other)."""
    Y, FT = mobility_inputs(100, 32, seed=0)
    ref, ref_abs = rpy.apply(Y, FT, with_abs=True, nthreads=8)
    out = {}
    for split in (1, 2):
        with fil.Filaments([32] * 100, precision=fil.FIL_PAIR32) as m:
            m.set_pair_schedule(128, 1, 2)
            m.set_source_split(split)
            VW = np.zeros_like(ref)
            m.mobility_apply(Y, FT, VW)
            VW2 = np.zeros_like(ref)
            m.mobility_apply(Y, FT, VW2)
            np.testing.assert_array_equal(VW, VW2)   # deterministic
        _check_mixed(VW, ref, ref_abs)
        out[split] = VW
    assert np.all(np.abs(out[1] - out[2]) <= 2 * C_MIXED * U32 * ref_abs)


def test_pair_schedule_rejections(fil):
    with fil.Filaments([32] * 4, precision=fil.FIL_PAIR32) as m:
        for bad in [(128, 2, 1), (512, 2, 1), (256, 4, 1), (256, 2, 0), (256, 2, 99), (64, 1, 1)]:
            with pytest.raises(fil.FilError) as e:
                m.set_pair_schedule(*bad)
            assert e.value.status == fil.FIL_EINVAL
        m.set_pair_schedule(128, 1, 2)
        assert m.pair_schedule() == (128, 1, 2)
        # the source split: 1 or 2, and 2 only with one target per thread
        for bad in (0, 3):
            with pytest.raises(fil.FilError) as e:
                m.set_source_split(bad)
            assert e.value.status == fil.FIL_EINVAL
        m.set_source_split(2)
        assert m.source_split() == 2
        m.set_pair_schedule(256, 2, 1)
        assert m.source_split() == 1          # a new schedule starts unsplit
        with pytest.raises(fil.FilError) as e:
            m.set_source_split(2)
        assert e.value.status == fil.FIL_EINVAL
    with fil.Filaments([32] * 4, precision=fil.FIL_FP64) as m:
        m.set_pair_schedule(128, 1, 1)
        with pytest.raises(fil.FilError) as e:
            m.set_source_split(2)             # the FP64 kernel has no split
        assert e.value.status == fil.FIL_EINVAL
