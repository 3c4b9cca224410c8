"""Compile the oracle's C sources into oracle/_lib (test infrastructure only).

The C oracle is built with plain -O2, no fast-math and no FMA contraction so
that it rounds the same way on x86-64 and AArch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "_lib")
SOURCES = {"liboracle_rpy.so": ["rpy.c"]}


def lib_path(name):
    return os.path.join(LIBDIR, name)


def build(force=False):
    os.makedirs(LIBDIR, exist_ok=True)
    for lib, srcs in SOURCES.items():
        out = lib_path(lib)
        src_paths = [os.path.join(HERE, s) for s in srcs]
        if (not force and os.path.exists(out)
                and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in src_paths)):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", out] + src_paths + ["-lm"]
        subprocess.check_call(cmd)


if __name__ == "__main__":
    build(force=True)
