"""Build the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain gcc, -O2 -ffp-contract=off so that no multiply-add is fused: the inside test
and the boundary fractions must be the IEEE operations written in the source.

The same source is also built with -fopenmp into oracle/liboracle_omp.so, the
multi-threaded CPU baseline (row and vector loops in static chunks, dot products summed
chunk by chunk in thread order).  Parity always uses the sequential build.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "saamg_oracle.c")
HDR = os.path.join(HERE, "saamg_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")

_FLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _compile(lib, extra, force):
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR), os.path.getmtime(__file__))
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    cmd = ["gcc"] + _FLAGS + extra + [SRC, "-o", lib + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the sequential oracle if it is missing or older than its sources."""
    return _compile(LIB, [], force)


def build_omp(force: bool = False):
    """Compile the OpenMP baseline build; None when the compiler has no OpenMP."""
    try:
        return _compile(LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        return None


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
