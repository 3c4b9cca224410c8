"""The allocation-free mobility apply (fil_rpy_apply_noalloc).

Some callers cannot allocate device memory -- for instance code running
inside another framework's memory pool, or in a process whose allocations
are owned by someone else -- so they cannot create a context. For them the
library offers one entry point whose scratch is a fixed static device array.
These tests check it through the C ABI on two calls in a row (the second on a
different input, so that whatever the first call left in the shared array
must not leak into the second):

* against the context-based fil_mobility_apply of a mixed-precision context:
  bit for bit, since both run the same three kernels with the same tile size
  and the same stream-K grid (min(resident CTAs x SMs, work units), which the
  static scratch holds in full on a 152-SM GB300), hence the same summation
  order;
* against the FP64 oracle within the mixed-precision bound the parity tests
  use (C_MIXED * 2^-24 * B per component);
* and that the second call leaves the device's free memory unchanged.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1903_12609_gb300.inputs import mobility_inputs

U32 = 2.0 ** -24
C_MIXED = 4 * 32 + 16


@pytest.fixture(scope="module")
def fil():
    from paper_1903_12609_gb300 import build
    build.build()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


def test_noalloc_rejects_sizes_beyond_the_maximum(fil):
    st = fil._lib.fil_rpy_apply_noalloc(32769, None, None, None, 1.0, 1.0, None)
    assert st == fil.FIL_EINVAL
    st = fil._lib.fil_rpy_apply_noalloc(0, None, None, None, 1.0, 1.0, None)
    assert st == fil.FIL_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_context_apply_and_oracle_on_two_calls(fil):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from oracle import rpy

    cases = [(mobility_inputs(100, 32, seed=21), [32] * 100, 1.0, 1.0),
             (mobility_inputs(37, 17, seed=22), [17] * 37, 1.3, 0.8)]
    for call, ((Y, FT), segs, a, eta) in enumerate(cases):
        S = Y.shape[0]
        Yd = torch.from_numpy(Y).cuda()
        FTd = torch.from_numpy(FT).cuda()
        with fil.Filaments(segs, a=a, eta=eta, precision=fil.FIL_MIXED) as m:
            ref = torch.empty((S, 6), dtype=torch.float64, device="cuda")
            m.mobility_apply(Yd, FTd, ref)
        out = torch.full((S, 6), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        fil.fil_rpy_apply_noalloc(S, Yd, FTd, out, a, eta)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:
            # the first call may load the library's device code (and with it the
            # static array); the second must not allocate anything
            assert free1 == free0, (free0, free1)
        got, ref = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        np.testing.assert_array_equal(got, ref)
        vw, B = rpy.apply(Y, FT, a, eta, with_abs=True, nthreads=8)
        err = np.abs(got - vw)
        assert np.all(err <= C_MIXED * U32 * B), float((err / B).max() / U32)


@pytest.mark.gpu
def test_noalloc_rejects_host_pointers(fil):
    pytest.importorskip("torch")
    Y, FT = mobility_inputs(2, 8, seed=23)
    VW = np.zeros((16, 6))
    st = fil._lib.fil_rpy_apply_noalloc(16, ctypes.c_void_p(Y.ctypes.data),
                                        ctypes.c_void_p(FT.ctypes.data),
                                        ctypes.c_void_p(VW.ctypes.data), 1.0, 1.0, None)
    assert st == fil.FIL_EINVAL
