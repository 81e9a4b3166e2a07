"""Build the FP64 oracle shared library (test infrastructure only).

`python oracle/build.py` compiles sbs_oracle.c with gcc into
oracle/_build/libsbs_oracle.so, and the same source again as C++ with a
counting double type (flop_count.cpp) into oracle/_build/libsbs_oracle_flops.so.
Floating-point contraction is disabled so the oracle evaluates every expression
exactly as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sbs_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsbs_oracle.so")
SRC_FLOPS = os.path.join(HERE, "flop_count.cpp")
LIB_FLOPS = os.path.join(OUT_DIR, "libsbs_oracle_flops.so")


def _stale(lib, srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(p) > os.path.getmtime(lib) for p in srcs)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or _stale(LIB, [SRC]):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def build_flops(force: bool = False) -> str:
    """The FLOP-counting build (single-threaded)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or _stale(LIB_FLOPS, [SRC, SRC_FLOPS]):
        cmd = ["g++", "-O1", "-std=c++17", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-Wno-unknown-pragmas", "-fPIC", "-shared", "-o", LIB_FLOPS + ".tmp", SRC_FLOPS, "-lm"]
        subprocess.check_call(cmd, cwd=HERE)
        os.replace(LIB_FLOPS + ".tmp", LIB_FLOPS)
    return LIB_FLOPS


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_flops(force="--force" in sys.argv))
