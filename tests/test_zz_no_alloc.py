"""The allocation-free mobility apply (fil_rpy_apply_noalloc).

Some callers cannot allocate device memory -- for instance code running
inside another framework's memory pool, or in a process whose allocations
are owned by someone else -- so they cannot create a context. For them the
library offers one entry point whose scratch is a fixed static device array.
These tests check it through the C ABI against the context-based
fil_mobility_apply (mixed precision) with the tolerance the mixed-precision
parity tests use, on two calls in a row (the second on a different input, so
that whatever the first call left in the shared array must not leak into the
second). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1903_12609_gb300.inputs import mobility_inputs

U32 = 2.0 ** -24
C_MIXED = 4 * 32 + 16


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_1903_12609_gb300 import fil
    st = fil._lib.fil_rpy_apply_noalloc(32769, None, None, None, 1.0, 1.0, None)
    assert st == fil.FIL_EINVAL
    st = fil._lib.fil_rpy_apply_noalloc(0, None, None, None, 1.0, 1.0, None)
    assert st == fil.FIL_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_context_apply_on_two_calls():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from oracle import rpy
    from paper_1903_12609_gb300 import fil

    cases = [(mobility_inputs(100, 32, seed=21), [32] * 100, 1.0, 1.0),
             (mobility_inputs(37, 17, seed=22), [17] * 37, 1.3, 0.8)]
    for (Y, FT), segs, a, eta in cases:
        S = Y.shape[0]
        Yd = torch.from_numpy(Y).cuda()
        FTd = torch.from_numpy(FT).cuda()
        with fil.Filaments(segs, a=a, eta=eta, precision=fil.FIL_MIXED) as m:
            ref = torch.empty((S, 6), dtype=torch.float64, device="cuda")
            m.mobility_apply(Yd, FTd, ref)
        out = torch.full((S, 6), float("nan"), dtype=torch.float64, device="cuda")
        fil.fil_rpy_apply_noalloc(S, Yd, FTd, out, a, eta)
        torch.cuda.synchronize()
        got, ref = out.cpu().numpy(), ref.cpu().numpy()
        _, B = rpy.apply(Y, FT, a, eta, with_abs=True, nthreads=8)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= C_MIXED * U32 * B)


@pytest.mark.gpu
def test_noalloc_rejects_host_pointers():
    torch = pytest.importorskip("torch")
    from paper_1903_12609_gb300 import fil
    Y, FT = mobility_inputs(2, 8, seed=23)
    VW = np.zeros((16, 6))
    st = fil._lib.fil_rpy_apply_noalloc(16, ctypes.c_void_p(Y.ctypes.data),
                                        ctypes.c_void_p(FT.ctypes.data),
                                        ctypes.c_void_p(VW.ctypes.data), 1.0, 1.0, None)
    assert st == fil.FIL_EINVAL
