"""Compile the CPU oracle (oracle.c) into oracle/liboracle.so.

Test infrastructure: the oracle is the plain CPU restatement the CUDA path is checked against.
Only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_P = os.path.join(HERE, "liboracle_p.so")  # the paper-like "_p" build (OpenMP on all host threads)
FLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall",
         "-Wno-unused-variable", "-Wno-unknown-pragmas"]


def _build(lib, extra, force):
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc"] + FLAGS + extra + ["-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Build liboracle.so (and, where the compiler has OpenMP, liboracle_p.so) if missing or
    older than oracle.c; return the path of liboracle.so."""
    _build(LIB, [], force)
    try:
        _build(LIB_P, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP: the "_p" baseline is then unavailable
    return LIB


def build_p(force: bool = False):
    """Path of liboracle_p.so, or None where it cannot be built."""
    build(force)
    return LIB_P if os.path.exists(LIB_P) else None


if __name__ == "__main__":
    print(build(force=True))
