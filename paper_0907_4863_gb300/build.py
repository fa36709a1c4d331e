"""Build libsaamg.so (the CUDA library behind include/saamg.h) in-tree for sm_103a.

One nvcc call per translation unit, run in parallel, then one link.  The geometry unit
is compiled with --fmad=false (the inside test and the boundary fractions must be the
plain IEEE operations of the source); host code is compiled with -ffp-contract=off.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsaamg.so")

UNITS = ["capi", "geometry", "stencil", "csr", "sell", "aggregate", "galerkin", "coarse", "pcg",
         "pic", "scan", "ktimer", "batch"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
          "-I" + INCLUDE, "-I" + CSRC]
PER_UNIT = {"geometry": ["--fmad=false"]}


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _headers():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + [
        os.path.join(INCLUDE, "saamg.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = _nvcc()
    headers = _headers()
    jobs = []
    for u in UNITS:
        src = os.path.join(CSRC, u + ".cu")
        obj = os.path.join(OBJDIR, u + ".o")
        if force or _stale(obj, [src] + headers + [__file__]):
            cmd = [nvcc] + ARCH + COMMON + PER_UNIT.get(u, []) + ["-c", src, "-o", obj]
            jobs.append((u, cmd))

    def run(job):
        u, cmd = job
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}.cu:\n{p.stderr}")
        return u

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    objs = [os.path.join(OBJDIR, u + ".o") for u in UNITS]
    if force or jobs or _stale(LIB, objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-cudart", "static"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n" + p.stderr)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
