"""Host-side arithmetic of bench.py (no GPU): the velocity-error summary of the
GPU apply against the oracle, and the pair-kernel roofline."""
import numpy as np

import bench


def test_velocity_error_summary():
    rng = np.random.default_rng(0)
    ref = rng.standard_normal((50, 6))
    B = np.abs(ref) + 1.0
    c = rng.uniform(0, 3, ref.shape)
    c[7, 2] = 9.5                                  # the worst component
    got = ref + c * bench.U32 * B * np.sign(rng.standard_normal(ref.shape))
    e = bench.velocity_error(got, ref, B)
    assert e["rows"] == 50
    assert abs(e["max_c"] - 9.5) < 1e-6
    assert abs(e["median_c"] - np.median(c)) < 1e-6
    assert e["within_bound"] and e["bound_c"] == 144
    assert abs(e["normwise"] - np.linalg.norm(got - ref) / np.linalg.norm(ref)) < 1e-15
    bad = got.copy()
    bad[3, 4] = ref[3, 4] + 200 * bench.U32 * B[3, 4]
    assert not bench.velocity_error(bad, ref, B)["within_bound"]


def test_pair_roofline_arithmetic():
    S = 32000.0
    r = bench.pair_roofline(S * S, pair_ms=10 * 1.7, n_launch=10)
    assert abs(r["avg_launch_ms"] - 1.7) < 1e-12
    want = 84 * S * S / 1.7e-3 / 1e12
    assert abs(r["achieved"] - want) < 1e-9
    assert abs(r["frac"] - want / bench.FP32_PEAK_TFLOPS) < 1e-12
    assert abs(bench.FP32_PEAK_TFLOPS - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"


def test_precision_names():
    class FakeFil:
        FIL_FP64, FIL_MIXED, FIL_PAIR32 = 0, 1, 2
    assert [bench.precision_code(FakeFil, n) for n in ("fp64", "mixed", "pair32")] == [0, 1, 2]
    assert set(bench.PRECISION_NOTE) == {"fp64", "mixed", "pair32"}
