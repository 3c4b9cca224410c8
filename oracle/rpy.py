"""ctypes wrapper of the C RPY oracle (oracle/rpy.c). Test infrastructure only.

Paper Sec. 2.7.1 (RPY mobility matrix); the overlapping-sphere branch is the
reading documented in rpy.c.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.lib_path("liboracle_rpy.so")
        if not os.path.exists(path):
            _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_rpy_pair_blocks.argtypes = [dp, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, dp, dp, dp, dp]
        lib.oracle_rpy_apply.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double,
                                         ctypes.c_double, dp, dp, ctypes.c_int]
        lib.oracle_rpy_apply_rows.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, ip, dp, dp,
                                              ctypes.c_int]
        _lib = lib
    return _lib


def _dp(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pair_blocks(d, same, a=1.0, eta=1.0):
    """The four 3x3 blocks (Mtt, Mtr, Mrt, Mrr) of one pair, d = Y_n - Y_m."""
    lib = _load()
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = [np.zeros((3, 3)) for _ in range(4)]
    lib.oracle_rpy_pair_blocks(_dp(d), int(bool(same)), float(a), float(eta),
                               *[_dp(o) for o in out])
    return tuple(out)


def apply(Y, FT, a=1.0, eta=1.0, with_abs=False, nthreads=1):
    """VW (S x 6) = M(Y) FT over all ordered pairs; optionally the magnitude sum."""
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(-1, 3)
    FT = np.ascontiguousarray(FT, dtype=np.float64).reshape(-1, 6)
    S = Y.shape[0]
    assert FT.shape[0] == S
    VW = np.zeros((S, 6))
    absVW = np.zeros((S, 6)) if with_abs else None
    lib.oracle_rpy_apply(S, _dp(Y), _dp(FT), float(a), float(eta), _dp(VW),
                         _dp(absVW) if with_abs else None, int(nthreads))
    return (VW, absVW) if with_abs else VW


def apply_rows(Y, FT, rows, a=1.0, eta=1.0, with_abs=False, nthreads=1):
    """Rows `rows` of the apply only (for sampled checks at full size)."""
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(-1, 3)
    FT = np.ascontiguousarray(FT, dtype=np.float64).reshape(-1, 6)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    S = Y.shape[0]
    out = np.zeros((rows.size, 6))
    aout = np.zeros((rows.size, 6)) if with_abs else None
    lib.oracle_rpy_apply_rows(S, _dp(Y), _dp(FT), float(a), float(eta), int(rows.size),
                              rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              _dp(out), _dp(aout) if with_abs else None, int(nthreads))
    return (out, aout) if with_abs else out
