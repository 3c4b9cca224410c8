"""Thin Python binding of the C ABI in include/fil.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: arrays are passed through as pointers. Arrays may be
numpy arrays (host memory) or torch CUDA tensors (device memory); both must be
C-contiguous float64 with the documented shapes. There is no fallback: if the
shared library is missing or does not load, importing the binding raises.

``Filaments`` is a small convenience wrapper that owns a context.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfil.so")

(FIL_OK, FIL_EINVAL, FIL_ENOMEM, FIL_ECUDA, FIL_ENOCONV, FIL_ENAN, FIL_ESTALL, FIL_ESTATE,
 FIL_EOVERFLOW) = range(9)
FIL_FP64, FIL_MIXED, FIL_PAIR32 = 0, 1, 2
FIL_J0_DRAG, FIL_J0_FILAMENT_RPY = 0, 1
FIL_EXTRAP_LINEAR, FIL_EXTRAP_QUADRATIC, FIL_EXTRAP_ADAPTIVE = 1, 2, 3
STATUS_NAMES = {0: "FIL_OK", 1: "FIL_EINVAL", 2: "FIL_ENOMEM", 3: "FIL_ECUDA", 4: "FIL_ENOCONV",
                5: "FIL_ENAN", 6: "FIL_ESTALL", 7: "FIL_ESTATE", 8: "FIL_EOVERFLOW"}

EXPORTED = ["fil_create", "fil_destroy", "fil_last_error", "fil_sizes", "fil_set_state",
            "fil_get_state", "fil_init_straight", "fil_set_external", "fil_mobility_apply",
            "fil_residual", "fil_broyden_begin", "fil_broyden_step", "fil_get_iterate",
            "fil_j0_solve", "fil_broyden_commit", "fil_step", "fil_set_dt", "fil_counters",
            "fil_profile", "fil_profile_read", "fil_rpy_apply_noalloc",
            "fil_mlp_create", "fil_mlp_destroy", "fil_mlp_set_params", "fil_mlp_get_params",
            "fil_mlp_set_norm", "fil_mlp_forward", "fil_mlp_gradients", "fil_mlp_train_step",
            "fil_tc_gemm_bf16", "fil_warm_features", "fil_warm_targets", "fil_warm_attach",
            "fil_warm_stats", "fil_create_ensemble", "fil_sys_stats", "fil_pair_count",
            "fil_set_graph", "fil_autotune", "fil_set_steric", "fil_set_tether",
            "fil_get_tether", "fil_fma_peak", "fil_set_j0_reuse", "fil_j0_stats",
            "fil_set_pair_schedule", "fil_pair_schedule", "fil_set_extrapolation",
            "fil_extrapolation", "fil_set_broyden_memory", "fil_set_source_split",
            "fil_source_split"]
MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_SEG = 800, 256, 192, 32
MLP_NPARAM = 256 * 800 + 256 + 2 * (256 * 256 + 256) + 192 * 256 + 192
FIL_WARM_BEST_OF_TWO, FIL_WARM_PREDICTION_FIRST = 0, 1


class FilError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class fil_params(ctypes.Structure):
    _fields_ = [("n_fil", ctypes.c_int32), ("seg_per_fil", ctypes.POINTER(ctypes.c_int32)),
                ("a", ctypes.c_double), ("eta", ctypes.c_double), ("dL", ctypes.c_double),
                ("KB", ctypes.c_double), ("KT", ctypes.c_double), ("gamma0", ctypes.c_double),
                ("kappa_mu", ctypes.c_double), ("kappa_nu", ctypes.c_double),
                ("dt", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("j0_model", ctypes.c_int32), ("stream", ctypes.c_void_p)]


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libfil.so not built at %s (run __graft_entry__.build())" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I64 = ctypes.POINTER(ctypes.c_int64)
    I32 = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "fil_create": [ctypes.POINTER(fil_params), ctypes.POINTER(P)],
        "fil_destroy": [P],
        "fil_last_error": [P],
        "fil_sizes": [P, I64, I64, I64],
        "fil_set_state": [P, P, P, P, P, P],
        "fil_get_state": [P, P, P, P, P, P],
        "fil_init_straight": [P, P, P, P, P],
        "fil_set_external": [P, P, P, P],
        "fil_mobility_apply": [P, P, P, P],
        "fil_residual": [P, P, P, D],
        "fil_broyden_begin": [P, D],
        "fil_broyden_step": [P, I32, D],
        "fil_get_iterate": [P, P, P],
        "fil_j0_solve": [P, P, P],
        "fil_broyden_commit": [P],
        "fil_step": [P, I32],
        "fil_set_dt": [P, ctypes.c_double],
        "fil_counters": [P, I64, I64, I64],
        "fil_profile": [P, ctypes.c_int32],
        "fil_profile_read": [P, I64, D],
        "fil_rpy_apply_noalloc": [ctypes.c_int64, P, P, P, ctypes.c_double, ctypes.c_double, P],
        "fil_fma_peak": [ctypes.c_int32, D, D],
        "fil_set_j0_reuse": [P, ctypes.c_int32],
        "fil_set_pair_schedule": [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
        "fil_pair_schedule": [P, I32, I32, I32],
        "fil_set_source_split": [P, ctypes.c_int32],
        "fil_source_split": [P, I32],
        "fil_j0_stats": [P, I64, I64],
        "fil_set_extrapolation": [P, ctypes.c_int32],
        "fil_set_broyden_memory": [P, ctypes.c_int32],
        "fil_extrapolation": [P, I32],
        "fil_mlp_create": [ctypes.c_int64, P, ctypes.POINTER(P)],
        "fil_mlp_destroy": [P],
        "fil_mlp_set_params": [P, P],
        "fil_mlp_get_params": [P, P],
        "fil_mlp_set_norm": [P, P, P, P, P],
        "fil_mlp_forward": [P, P, P, ctypes.c_int64],
        "fil_mlp_gradients": [P, P, P, ctypes.c_int64, P, ctypes.POINTER(ctypes.c_float)],
        "fil_mlp_train_step": [P, P, P, ctypes.c_int64, ctypes.c_float,
                               ctypes.POINTER(ctypes.c_float)],
        "fil_tc_gemm_bf16": [P, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P],
        "fil_warm_features": [P, P],
        "fil_warm_targets": [P, P],
        "fil_warm_attach": [P, P, ctypes.c_int32],
        "fil_warm_stats": [P, I64, I64, I64],
        "fil_create_ensemble": [ctypes.POINTER(fil_params), ctypes.c_int32, I32,
                                ctypes.POINTER(P)],
        "fil_sys_stats": [P, I32, D],
        "fil_pair_count": [P, D],
        "fil_set_graph": [P, ctypes.c_int32],
        "fil_autotune": [P, ctypes.c_int32, I32, I32, D],
        "fil_set_steric": [P, ctypes.c_double, ctypes.c_double],
        "fil_set_tether": [P, P, P, P],
        "fil_get_tether": [P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None if name in ("fil_destroy", "fil_mlp_destroy") else (
            ctypes.c_char_p if name == "fil_last_error" else ctypes.c_int)
    return lib


_lib = load_library()


def _ptr(a, dtype="float64"):
    """Device or host address of a C-contiguous array of `dtype` (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):                       # torch tensor
        if str(a.dtype) != "torch." + dtype or not a.is_contiguous():
            raise TypeError("torch tensors must be contiguous " + dtype)
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.dtype(dtype) and a.flags["C_CONTIGUOUS"]):
        raise TypeError("numpy arrays must be C-contiguous " + dtype)
    return ctypes.c_void_p(a.ctypes.data)


def _check(ctx, status):
    if status != FIL_OK:
        msg = _lib.fil_last_error(ctx) if ctx else b""
        raise FilError(status, (msg or b"").decode())


# ---- functions with the names of the C entry points ------------------------

def fil_create(seg_per_fil, a=1.0, eta=1.0, dL=2.2, KB=1.0, KT=1.0, gamma0=0.0, kappa_mu=0.0,
               kappa_nu=0.0, dt=0.01, tol=1e-8, max_iter=50, precision=FIL_FP64,
               j0_model=FIL_J0_DRAG, stream=None):
    segs = np.ascontiguousarray(seg_per_fil, dtype=np.int32)
    p = fil_params(int(segs.size), segs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), a, eta, dL,
                   KB, KT, gamma0, kappa_mu, kappa_nu, dt, tol, int(max_iter), int(precision),
                   int(j0_model), ctypes.c_void_p(stream) if stream else None)
    ctx = ctypes.c_void_p()
    _check(None, _lib.fil_create(ctypes.byref(p), ctypes.byref(ctx)))
    return ctx


def fil_create_ensemble(seg_per_fil, fil_per_sys, a=1.0, eta=1.0, dL=2.2, KB=1.0, KT=1.0,
                        gamma0=0.0, kappa_mu=0.0, kappa_nu=0.0, dt=0.01, tol=1e-8, max_iter=50,
                        precision=FIL_FP64, j0_model=FIL_J0_DRAG, stream=None):
    segs = np.ascontiguousarray(seg_per_fil, dtype=np.int32)
    fps = np.ascontiguousarray(fil_per_sys, dtype=np.int32)
    p = fil_params(int(segs.size), segs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), a, eta, dL,
                   KB, KT, gamma0, kappa_mu, kappa_nu, dt, tol, int(max_iter), int(precision),
                   int(j0_model), ctypes.c_void_p(stream) if stream else None)
    ctx = ctypes.c_void_p()
    _check(None, _lib.fil_create_ensemble(ctypes.byref(p), int(fps.size),
                                          fps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          ctypes.byref(ctx)))
    return ctx


def fil_sys_stats(ctx, n_sys):
    it = np.zeros(n_sys, dtype=np.int32)
    fi = np.zeros(n_sys)
    _check(ctx, _lib.fil_sys_stats(ctx, it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   fi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return it, fi


def fil_autotune(ctx, reps=3):
    tile, ctas, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(ctx, _lib.fil_autotune(ctx, int(reps), ctypes.byref(tile), ctypes.byref(ctas),
                                  ctypes.byref(ms)))
    return tile.value, ctas.value, ms.value


def fil_set_pair_schedule(ctx, tile, targets_per_thread, ctas_per_sm):
    _check(ctx, _lib.fil_set_pair_schedule(ctx, int(tile), int(targets_per_thread),
                                           int(ctas_per_sm)))


def fil_pair_schedule(ctx):
    t, p, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, _lib.fil_pair_schedule(ctx, ctypes.byref(t), ctypes.byref(p), ctypes.byref(c)))
    return t.value, p.value, c.value


def fil_set_source_split(ctx, split):
    _check(ctx, _lib.fil_set_source_split(ctx, int(split)))


def fil_source_split(ctx):
    v = ctypes.c_int32()
    _check(ctx, _lib.fil_source_split(ctx, ctypes.byref(v)))
    return v.value


def fil_set_graph(ctx, enable):
    _check(ctx, _lib.fil_set_graph(ctx, int(bool(enable))))


def fil_set_steric(ctx, FS, chi=1.1):
    _check(ctx, _lib.fil_set_steric(ctx, float(FS), float(chi)))


def fil_set_tether(ctx, mask, Y1=None, u1=None):
    """mask: sequence of M flags (None unties every filament); Y1, u1: (M, 3)."""
    if mask is None:
        _check(ctx, _lib.fil_set_tether(ctx, None, None, None))
        return
    m = np.ascontiguousarray(np.asarray(mask).astype(np.int32))
    _check(ctx, _lib.fil_set_tether(ctx, _ptr(m, "int32"), _ptr(Y1), _ptr(u1)))


def fil_get_tether(ctx, lam):
    _check(ctx, _lib.fil_get_tether(ctx, _ptr(lam)))


def fil_pair_count(ctx):
    v = ctypes.c_double()
    _check(ctx, _lib.fil_pair_count(ctx, ctypes.byref(v)))
    return v.value


def fil_destroy(ctx):
    _lib.fil_destroy(ctx)


def fil_last_error(ctx):
    return (_lib.fil_last_error(ctx) or b"").decode()


def fil_sizes(ctx):
    s, x, l = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, _lib.fil_sizes(ctx, ctypes.byref(s), ctypes.byref(x), ctypes.byref(l)))
    return s.value, x.value, l.value


def fil_set_state(ctx, Y, q, Yprev=None, u=None, Lambda=None):
    _check(ctx, _lib.fil_set_state(ctx, _ptr(Y), _ptr(q), _ptr(Yprev), _ptr(u), _ptr(Lambda)))


def fil_get_state(ctx, Y=None, q=None, Yprev=None, u=None, Lambda=None):
    _check(ctx, _lib.fil_get_state(ctx, _ptr(Y), _ptr(q), _ptr(Yprev), _ptr(u), _ptr(Lambda)))


def fil_init_straight(ctx, base, t, mu, xi=None):
    _check(ctx, _lib.fil_init_straight(ctx, _ptr(base), _ptr(t), _ptr(mu), _ptr(xi)))


def fil_set_external(ctx, Fext=None, Text=None, follower=None):
    _check(ctx, _lib.fil_set_external(ctx, _ptr(Fext), _ptr(Text), _ptr(follower)))


def fil_mobility_apply(ctx, Y, FT, VW):
    _check(ctx, _lib.fil_mobility_apply(ctx, _ptr(Y), _ptr(FT), _ptr(VW)))


def fil_residual(ctx, X, f):
    finf = ctypes.c_double()
    _check(ctx, _lib.fil_residual(ctx, _ptr(X), _ptr(f), ctypes.byref(finf)))
    return finf.value


def fil_broyden_begin(ctx):
    finf = ctypes.c_double()
    _check(ctx, _lib.fil_broyden_begin(ctx, ctypes.byref(finf)))
    return finf.value


def fil_broyden_step(ctx):
    conv, finf = ctypes.c_int32(), ctypes.c_double()
    _check(ctx, _lib.fil_broyden_step(ctx, ctypes.byref(conv), ctypes.byref(finf)))
    return bool(conv.value), finf.value


def fil_get_iterate(ctx, X=None, f=None):
    _check(ctx, _lib.fil_get_iterate(ctx, _ptr(X), _ptr(f)))


def fil_j0_solve(ctx, b, x):
    _check(ctx, _lib.fil_j0_solve(ctx, _ptr(b), _ptr(x)))


def fil_broyden_commit(ctx):
    _check(ctx, _lib.fil_broyden_commit(ctx))


def fil_step(ctx):
    it = ctypes.c_int32()
    _check(ctx, _lib.fil_step(ctx, ctypes.byref(it)))
    return it.value


def fil_set_dt(ctx, dt):
    _check(ctx, _lib.fil_set_dt(ctx, float(dt)))


def fil_set_j0_reuse(ctx, max_age):
    _check(ctx, _lib.fil_set_j0_reuse(ctx, int(max_age)))


def fil_j0_stats(ctx):
    b, r = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, _lib.fil_j0_stats(ctx, ctypes.byref(b), ctypes.byref(r)))
    return b.value, r.value


def fil_set_extrapolation(ctx, order):
    _check(ctx, _lib.fil_set_extrapolation(ctx, int(order)))


def fil_set_broyden_memory(ctx, keep):
    _check(ctx, _lib.fil_set_broyden_memory(ctx, int(keep)))


def fil_extrapolation(ctx):
    o = ctypes.c_int32()
    _check(ctx, _lib.fil_extrapolation(ctx, ctypes.byref(o)))
    return o.value


def fil_counters(ctx):
    a, b, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, _lib.fil_counters(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k)))
    return a.value, b.value, k.value


def fil_profile(ctx, enable):
    _check(ctx, _lib.fil_profile(ctx, int(bool(enable))))


def fil_profile_read(ctx):
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(ctx, _lib.fil_profile_read(ctx, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def fil_rpy_apply_noalloc(n_seg, Y, FT, VW, a=1.0, eta=1.0, stream=None):
    """Context-free mixed-precision RPY apply that allocates nothing (device
    arrays only; see include/fil.h for the limits and the sharing rules)."""
    st = _lib.fil_rpy_apply_noalloc(int(n_seg), _ptr(Y), _ptr(FT), _ptr(VW), float(a),
                                    float(eta), ctypes.c_void_p(stream) if stream else None)
    if st != FIL_OK:
        raise FilError(st, "fil_rpy_apply_noalloc")


def fil_fma_peak(fp64=False):
    """Measured FMA rate of the current device: (flops/s, SM MHz during the
    run), packed FP32x2 FMAs or FP64 FMAs at full occupancy."""
    fl, mhz = ctypes.c_double(), ctypes.c_double()
    st = _lib.fil_fma_peak(1 if fp64 else 0, ctypes.byref(fl), ctypes.byref(mhz))
    if st != FIL_OK:
        raise FilError(st, "fil_fma_peak")
    return fl.value, mhz.value


# ---- warm-start network (include/fil_mlp.h); FP32 arrays ---------------------

def _f32(a):
    return _ptr(a, "float32")


def fil_mlp_create(max_batch, stream=None):
    m = ctypes.c_void_p()
    _check(None, _lib.fil_mlp_create(int(max_batch), ctypes.c_void_p(stream) if stream else None,
                                     ctypes.byref(m)))
    return m


def fil_mlp_destroy(m):
    _lib.fil_mlp_destroy(m)


def fil_mlp_set_params(m, params):
    _check(None, _lib.fil_mlp_set_params(m, _f32(params)))


def fil_mlp_get_params(m, params):
    _check(None, _lib.fil_mlp_get_params(m, _f32(params)))


def fil_mlp_set_norm(m, in_mean, in_std, out_mean, out_std):
    _check(None, _lib.fil_mlp_set_norm(m, _f32(in_mean), _f32(in_std), _f32(out_mean),
                                       _f32(out_std)))


def fil_mlp_forward(m, x, y, batch):
    _check(None, _lib.fil_mlp_forward(m, _f32(x), _f32(y), int(batch)))


def fil_mlp_gradients(m, x, target, batch, grad):
    loss = ctypes.c_float()
    _check(None, _lib.fil_mlp_gradients(m, _f32(x), _f32(target), int(batch), _f32(grad),
                                        ctypes.byref(loss)))
    return loss.value


def fil_mlp_train_step(m, x, target, batch, lr):
    loss = ctypes.c_float()
    _check(None, _lib.fil_mlp_train_step(m, _f32(x), _f32(target), int(batch), float(lr),
                                         ctypes.byref(loss)))
    return loss.value


def fil_tc_gemm_bf16(A, lda, B, ldb, C, ldc, M, N, K, stream=None):
    """A, B: uint16 (BF16 bit patterns) device tensors viewed as int16; C float32."""
    _check(None, _lib.fil_tc_gemm_bf16(_ptr(A, "int16"), int(lda), _ptr(B, "int16"), int(ldb),
                                       _f32(C), int(ldc), int(M), int(N), int(K),
                                       ctypes.c_void_p(stream) if stream else None))


def fil_warm_features(ctx, feat):
    _check(ctx, _lib.fil_warm_features(ctx, _f32(feat)))


def fil_warm_targets(ctx, targ):
    _check(ctx, _lib.fil_warm_targets(ctx, _f32(targ)))


def fil_warm_attach(ctx, net, mode=FIL_WARM_BEST_OF_TWO):
    _check(ctx, _lib.fil_warm_attach(ctx, net, int(mode)))


def fil_warm_stats(ctx):
    a, b, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, _lib.fil_warm_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(r)))
    return a.value, b.value, r.value


class Filaments:
    """Owns one context; methods forward to the fil_* functions above."""

    def __init__(self, seg_per_fil, fil_per_sys=None, **params):
        if fil_per_sys is None:
            self.ctx = fil_create(seg_per_fil, **params)
            self.n_sys = 1
        else:
            self.ctx = fil_create_ensemble(seg_per_fil, fil_per_sys, **params)
            self.n_sys = len(fil_per_sys)
        self.S, self.nX, self.nlam = fil_sizes(self.ctx)
        self.M = len(seg_per_fil)

    def sys_stats(self):
        return fil_sys_stats(self.ctx, self.n_sys)

    def close(self):
        if self.ctx is not None:
            fil_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __getattr__(self, name):
        if name.startswith("__"):
            raise AttributeError(name)
        fn = globals().get("fil_" + name)
        if fn is None:
            raise AttributeError(name)
        return lambda *a, **k: fn(self.ctx, *a, **k)
