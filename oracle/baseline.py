"""Time the FP64 CPU oracle on this host's cores (the CPU baseline; test infrastructure).

Each pass is the whole method on one seeded right-hand side: build the operator, set up the
hierarchy, PCG to the tolerance.  Build, setup and solve are timed separately.  The
sequential build is the parity oracle itself; with --openmp the same source built with
-fopenmp runs on --threads threads (default: every core this process may use).

    python -m oracle.baseline --workload pipe --n 256 --mode linear --passes 3 [--openmp]

prints one JSON object: the per-pass records and their means.  With --solve cases.json
--out sol.npz it writes the oracle's solutions of the listed cases instead (the error of a
GPU result against the oracle).  Run it as its own process:
the library choice (sequential or OpenMP) is made when the oracle is first loaded.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MODES = {"constant": 0, "linear": 1, "quadratic": 2}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def workload(kind, n, mode):
    from paper_0907_4863_gb300 import inputs as I
    if kind == "pipe":
        return I.pipe_workload(n, mode)
    if kind == "cylinder":
        return I.cylinder_workload(n, mode)
    raise ValueError(kind)


def run_passes(w, passes, rtol=1e-8, max_coarse=4096, max_levels=10, beta_rule=0, seed0=0,
               on_pass=None):
    from oracle import oracle as O
    from paper_0907_4863_gb300 import inputs as I
    d, g = w.domain, w.grid
    recs = []
    for k in range(passes):
        rho = I.gaussian_bunch(g, w.centre, w.sigma, seed=seed0 + k)
        t0 = time.perf_counter()
        op = O.Operator(g.n, g.h, g.origin, d.a, d.b, d.taper, d.cx, d.cy, d.zbc, d.symmetrize,
                        w.mode)
        t1 = time.perf_counter()
        h = O.Hierarchy(op, max_coarse=max_coarse, max_levels=max_levels)
        t2 = time.perf_counter()
        _, info = h.solve(rho, rtol=rtol, beta_rule=beta_rule)
        t3 = time.perf_counter()
        rec = {"build_s": t1 - t0, "setup_s": t2 - t1, "solve_s": t3 - t2, "total_s": t3 - t0,
               "iters": info["iters"], "relres_true": info["relres_true"],
               "unknowns": op.n, "levels": [h.n(l) for l in range(h.levels)]}
        recs.append(rec)
        if on_pass:
            on_pass(rec)
        del h, op
    return recs


def workload_to_dict(w):
    import dataclasses
    return dataclasses.asdict(w)


def workload_from_dict(d):
    from paper_0907_4863_gb300 import inputs as I
    return I.Workload(d["name"], I.Grid(tuple(d["grid"]["n"]), tuple(d["grid"]["h"]),
                                        tuple(d["grid"]["origin"])),
                      I.Domain(**d["domain"]), d["mode"], sigma=tuple(d["sigma"]),
                      centre=tuple(d["centre"]), jitter=d["jitter"])


def solve_cases(cases):
    """Oracle solutions of a list of cases: {"workload": dict, "seed": s (Gaussian bunch of
    that seed), "rtol": [r, ...], "beta_rule": b, "cheb_degree": d, "max_coarse": m}.  One
    hierarchy per distinct (workload, degree, max_coarse); returns a dict of box arrays keyed
    "<case index>_<rtol index>", and the iteration counts."""
    from oracle import oracle as O
    from paper_0907_4863_gb300 import inputs as I
    hs, sols, iters = {}, {}, {}
    for k, c in enumerate(cases):
        w = workload_from_dict(c["workload"])
        key = (w.name, c.get("cheb_degree", 2), c.get("max_coarse", 4096))
        if key not in hs:
            d, g = w.domain, w.grid
            op = O.Operator(g.n, g.h, g.origin, d.a, d.b, d.taper, d.cx, d.cy, d.zbc,
                            d.symmetrize, w.mode)
            hs.clear()  # one hierarchy at a time (memory)
            hs[key] = O.Hierarchy(op, cheb_degree=key[1], max_coarse=key[2])
        rho = I.gaussian_bunch(w.grid, w.centre, w.sigma, c["seed"])
        for j, rtol in enumerate(c["rtol"]):
            x, info = hs[key].solve(rho, rtol=rtol, beta_rule=c.get("beta_rule", 0))
            sols[f"{k}_{j}"] = x
            iters[f"{k}_{j}"] = info["iters"]
    return sols, iters


def summary(recs):
    keys = ("build_s", "setup_s", "solve_s", "total_s")
    out = {k: sum(r[k] for r in recs) / len(recs) for k in keys}
    out["solves_per_s"] = len(recs) / sum(r["total_s"] for r in recs)
    out["iters"] = [r["iters"] for r in recs]
    out["unknowns"] = recs[0]["unknowns"]
    out["levels"] = recs[0]["levels"]
    out["relres_true_max"] = max(r["relres_true"] for r in recs)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="pipe", choices=["pipe", "cylinder"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--mode", default="linear", choices=list(MODES))
    ap.add_argument("--passes", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--max-coarse", type=int, default=4096)
    ap.add_argument("--max-levels", type=int, default=10)
    ap.add_argument("--openmp", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--solve", default=None, help="JSON file of cases: write their solutions")
    ap.add_argument("--out", default=None, help="output .npz of --solve")
    a = ap.parse_args()
    threads = 1
    if a.openmp:
        threads = a.threads or host_cores()
        os.environ["SAAMG_ORACLE_OPENMP"] = "1"
        os.environ["OMP_NUM_THREADS"] = str(threads)
    if a.solve:
        import numpy as np
        t0 = time.perf_counter()
        sols, iters = solve_cases(json.load(open(a.solve)))
        np.savez(a.out, **sols)
        print(json.dumps({"iters": iters, "seconds": time.perf_counter() - t0, "threads": threads}),
              flush=True)
        return
    w = workload(a.workload, a.n, MODES[a.mode])
    if a.warmup:
        run_passes(w, a.warmup, a.rtol, a.max_coarse, a.max_levels, seed0=1000)
    recs = run_passes(w, a.passes, a.rtol, a.max_coarse, a.max_levels)
    out = {"workload": w.name, "mode": a.mode, "rtol": a.rtol, "build": "openmp" if a.openmp else "sequential",
           "threads": threads, "host_cores": host_cores(), "passes": recs, **summary(recs)}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
