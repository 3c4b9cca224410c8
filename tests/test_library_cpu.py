"""CPU-side checks of the C-ABI library: it loads, exports every entry point
that include/*.h declare, and rejects invalid parameters before touching
the GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fil_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1903_12609_gb300 import build
    build.build()
    from paper_1903_12609_gb300 import fil
    return fil


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib._lib, n), n
    assert sorted(lib.EXPORTED) == names


@pytest.mark.parametrize("bad", [dict(a=0.0), dict(eta=-1.0), dict(dL=0.0), dict(dt=0.0),
                                 dict(tol=0.0), dict(max_iter=0), dict(precision=7), dict(precision=3),
                                 dict(KB=float("nan"))])
def test_invalid_parameters_are_rejected_on_the_host(lib, bad):
    with pytest.raises(lib.FilError) as e:
        lib.fil_create([4, 4], **bad)
    assert e.value.status == lib.FIL_EINVAL


def test_invalid_layout_is_rejected(lib):
    for segs in ([], [3, 0], [-1]):
        with pytest.raises(lib.FilError) as e:
            lib.fil_create(segs)
        assert e.value.status == lib.FIL_EINVAL


def test_fma_peak_rejects_an_unknown_precision(lib):
    import ctypes
    fl, mhz = ctypes.c_double(), ctypes.c_double()
    assert lib._lib.fil_fma_peak(2, ctypes.byref(fl), ctypes.byref(mhz)) == lib.FIL_EINVAL


def test_oracle_library_builds():
    from oracle import build
    build.build()
    assert os.path.exists(build.lib_path("liboracle_rpy.so"))
    ctypes.CDLL(build.lib_path("liboracle_rpy.so"))


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: importing the binding from a copy of the package that
    has no built library raises ImportError."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_1903_12609_gb300")
    shutil.copytree(pkg, tmp_path / "paper_1903_12609_gb300",
                    ignore=shutil.ignore_patterns("_lib", "weights", "__pycache__"))
    env = dict(os.environ, PYTHONPATH=str(tmp_path))
    r = subprocess.run([sys.executable, "-c", "import paper_1903_12609_gb300.fil"],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libfil.so" in r.stderr
