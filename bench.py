#!/usr/bin/env python
"""SAAMG-PCG benchmark: solves/s to relative residual 1e-8 on the 256^3 elliptic pipe.

One step = one pass of the whole method on a new seeded Gaussian-bunch charge density:
build the operator (inside test, boundary rows, scaling), set up the SA-AMG hierarchy
(MIS-2 aggregation, prolongators, Galerkin products, coarse LU) and solve with PCG to
||r|| <= 1e-8 ||b||.  Prints one JSON line with the throughput, the end-to-end figure through
the host-buffer call, the roofline of the dominant kernel, clocks, the CPU baseline and the
mixed-precision, batched and serving legs.  --impl reference times the FP64 CPU oracle instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0907_4863_gb300 import inputs as I  # noqa: E402

RTOL = 1e-8
METRIC = "solves/s to rel-residual 1e-8 at 256^3 (mixed/batched vs FP64 GPU); HBM GB/s; p99"
UNIT = "solves/s"
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the FP64 level-0 Chebyshev step
# on the 256^3 elliptic pipe, from its ncu capture; None for other kernels or sizes, and to be
# reset whenever that kernel changes
# (class, precision, n) -> DRAM bytes per launch (ncu, dram__bytes_read + dram__bytes_write); the
# BF16 mode's level-0 passes are the FP32 kernels
TRAFFIC_BYTES = {("stencil_smooth", 0, 256): 364.0e6,
                 ("stencil_smooth", 1, 256): 125.1e6, ("stencil_smooth", 2, 256): 125.1e6,
                 ("stencil_resid", 1, 256): 82.5e6, ("stencil_resid", 2, 256): 82.5e6,
                 ("prolong0", 1, 256): 81.3e6, ("prolong0", 2, 256): 81.3e6}
# kernel timing classes of the solve phase (one kernel template each)
SOLVE_CLASSES = ("stencil_smooth", "stencil_apply", "stencil_resid", "stencil_first",
                 "coarse_csr", "coarse_deep", "transfer", "transfer_deep", "prolong0")


def fp64_peak(device=0, sm_max_mhz=None):
    """FP64 issue roof of the device: SMs x 2 FP64 FMA per clock x 2 flop x maximum SM clock.
    The SM count is the device's own; the clock is the maximum nvidia-smi reported during the
    run, else the one recorded with the measured peaks, else GB300's 2070 MHz."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    if not sm_max_mhz:
        path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        peaks = json.load(open(path)) if os.path.exists(path) else {}
        sm_max_mhz = peaks.get("sm_max_mhz", 2070.0)
    return {"tflops": sms * 2 * 2 * sm_max_mhz * 1e6 / 1e12,
            "source": f"derived: {sms} SMs x 2 FP64 FMA/clk x 2 flop x {sm_max_mhz:.0f} MHz"}


FP64_PEAK = {"tflops": 152 * 2 * 2 * 2.07e9 / 1e12, "source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="grid size of the elliptic pipe workload")
    ap.add_argument("--precision", choices=list(PREC), default="fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the mixed-precision and reuse legs")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (64 instances) leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default level-0 stencil launch shapes")
    ap.add_argument("--leg", choices=["batched", "serving"], default=None,
                    help="run only this leg and print its JSON (no headline line)")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the 10,000-request serving stream to replay")
    return ap.parse_args()


def workload(n):
    w = I.pipe_workload(n, I.LINEAR)
    return w


def max_over_ranks(x, world, device):
    """The slowest rank's value (replicas: the job ends with its last rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, seconds):
    """Solves per second of the whole job: every replica completes `steps` solves."""
    return world * steps / seconds


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# Level-0 stencil launch shapes chosen by the autotuner for the workload (precision 0: FP64
# passes, 1: FP32), applied to every operator the bench builds for it.
SHAPES = {}


def shaped_operator(S, dom, grid, mode):
    op = S.build_operator(dom, grid, mode)
    for sp, cfg in SHAPES.items():
        S.set_stencil_config(op, sp, cfg)
    return op


def tune_shapes(S, dom, grid, mode):
    """Autotunes the level-0 stencil launch shape of both precisions once per workload."""
    op = S.build_operator(dom, grid, mode)
    out = {}
    for sp in (0, 1):
        default = S.stencil_config(op, sp)
        best, us = S.autotune_stencil(op, sp)
        S.set_stencil_config(op, sp, default)
        SHAPES[sp] = best
        out["fp64" if sp == 0 else "fp32"] = {"default": default, "chosen": best,
                                              "chebyshev_step_us": us}
    op.free()
    return out


def run_ours(args):
    import torch
    from paper_0907_4863_gb300 import saamg as S

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    S.use_torch_allocator()
    w = workload(args.n)
    dom, grid = S.make_domain(w.domain), S.make_grid(w.grid)
    prec = PREC[args.precision]
    params = S.params_default(max_coarse=4096, precision=prec, beta_rule=1 if prec else 0)
    nsteps = args.warmup + args.steps
    # every step gets its own seeded right-hand side, resident in HBM before timing
    rhs = [torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=1000 * rank + k)).cuda()
           for k in range(nsteps)]
    phis = [torch.zeros_like(r) for r in rhs]
    stream = torch.cuda.current_stream()
    infos = []
    # once per workload, before the warm-up steps (like any autotuned kernel)
    shapes = None if args.no_autotune else tune_shapes(S, dom, grid, w.mode)

    def step(k):
        op = shaped_operator(S, dom, grid, w.mode)
        h = S.setup(op, params)
        phis[k].zero_()
        info = S.solve(h, rhs[k], phis[k], rtol=RTOL)
        infos.append((info, h.info()))
        h.free()
        op.free()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for k in range(args.warmup):
        step(k)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    launches0 = S.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    e0.record(stream)
    for k in range(args.warmup, nsteps):
        step(k)
    e1.record(stream)
    barrier()
    t_host = time.perf_counter() - t_host0
    launches = S.kernel_launches() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    # Per-class kernel times: the solve's kernels run inside the device-loop graph, where no
    # event can be recorded per launch, so the same steps are repeated with the host-driven
    # loop (device_loop = 0: the same kernels in the same order, the same bits) and a CUDA
    # event pair around every launch of the timed classes, on the launching stream.
    params_t = S.params_default(max_coarse=4096, precision=prec, beta_rule=1 if prec else 0,
                                device_loop=0)
    S.kernel_timing(True)
    for c in range(len(S.KT_NAMES)):
        S.kernel_timing_read(c)
    for k in range(args.warmup, nsteps):
        op_t = shaped_operator(S, dom, grid, w.mode)
        h_t = S.setup(op_t, params_t)
        phis[k].zero_()
        S.solve(h_t, rhs[k], phis[k], rtol=RTOL)
        h_t.free()
        op_t.free()
    torch.cuda.synchronize()
    S.kernel_timing(False)
    ktime = {S.KT_NAMES[c]: S.kernel_timing_read(c) for c in range(len(S.KT_NAMES))}
    timed = infos[args.warmup:]
    iters = [i["iters"] for i, _ in timed]
    relres = max(i["relres_true"] for i, _ in timed)
    assert all(i["converged"] == 1 for i, _ in timed), "a timed solve did not converge"
    hinfo = timed[-1][1]
    value = whole_job_rate(world, args.steps, ms / 1e3)

    # --- roofline of the dominant kernel (live, CUDA events on the launching stream).  Each
    # solve-phase class is one kernel template; the sparse products of the setup are several
    # different kernels, reported as a class time only.
    FP64_PEAK.update(fp64_peak(local, clk.get("sm_max_mhz")))
    dom_name = max(SOLVE_CLASSES, key=lambda k: ktime[k][0])
    ib1 = level1_index_bytes(hinfo)
    roof = roofline(dom_name, ktime[dom_name], prec, args.n, ib1)
    if roof:
        roof["measured_on"] = ("CUDA events around every launch on its stream, in a repeat of "
                               "the timed steps on the host-driven PCG loop (same kernels)")

    # --- end to end through the public API with host buffers (pinned), copies in the region
    nbox = w.grid.nbox
    host_rho = [torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=5000 + k)).pin_memory()
                for k in range(args.steps)]
    host_phi = torch.zeros(nbox, dtype=torch.float64).pin_memory()

    def e2e_step(k):
        op = shaped_operator(S, dom, grid, w.mode)
        h = S.setup(op, params)
        host_phi.zero_()
        info = S.solve_host(h, host_rho[k].numpy(), host_phi.numpy(), rtol=RTOL)
        assert info["converged"] == 1
        h.free()
        op.free()

    e2e_step(0)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    barrier()
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e = {"value": whole_job_rate(world, args.steps, t_e2e), "unit": UNIT,
           "h2d_bytes_per_step": 2 * nbox * 8, "d2h_bytes_per_step": nbox * 8}

    extra = {}
    if not args.no_extra:
        extra = extra_legs(S, torch, w, dom, grid, rhs[args.warmup], args)
        extra.update(mixed_quadratic_leg(S, torch, args))
        extra["aggregation_cubes_vs_mis2"] = aggregation_leg(S, torch, args)
        extra["coarse_gauss_seidel_vs_lu"] = coarse_solver_leg(S, torch, args)
        extra["pic_transfers"] = pic_leg(S, torch, args)
        extra["grid_sizes"] = sizes_leg(S, torch)
    del rhs, phis
    torch.cuda.empty_cache()
    if not args.no_batched:
        extra["batched_c4"] = batched_leg(S, torch)
    if not args.no_serve:
        extra["serving_c5"] = serving_leg(S, torch, args.serve_requests)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32+f64",
        "data": "synthetic (seeded Gaussian bunch, no dataset)",
        "config": {"workload": f"{w.name}, linear extrapolation, Robin ends, rtol 1e-8, coarse <= 4096, "
                               f"{args.precision} V-cycle; step = build operator + AMG setup + PCG solve",
                   "grid": list(w.grid.n), "unknowns": hinfo["n"][0], "levels": hinfo["n"],
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (rho 134 MB, hierarchy > 1 GB)"},
        "iters": iters, "relres_true_max": relres,
        "host_wall_ms_per_step": 1e3 * t_host / args.steps,
        "kernel_classes_ms_per_step": {k: v[0] / args.steps for k, v in ktime.items()},
        "roofline": roof, "clocks": clk, "gpu_launches": launches, "e2e": e2e,
        "stencil_shape_autotune": shapes,
    }
    out.update(extra)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.n)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def roofline(name, rec, prec, n=256, index_bytes=4):
    """Algorithmic work per launch / average launch duration of one timing class.

    Stencil classes count rows; the sparse-matrix classes (coarse_csr, transfer) count
    matrix entries.  FP64 passes are FP64-issue-bound on this part and are reported against
    the derived FP64 peak; the FP32/BF16 passes against the measured HBM copy bandwidth.
    """
    total_ms, launches, units = rec
    if launches == 0 or total_ms <= 0:
        return None
    avg_s = total_ms / launches / 1e3
    per = units / launches
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    if name == "stencil_apply":
        prec = 0  # the CG product A p is FP64 in every precision mode
    w = 8 if prec == 0 else 4
    if name == "prolong0":
        # matrix-free level-0 prolongation (FP32 V-cycle): per row the aggregate index and
        # x in / x out; 2 flops per coupling of the 7-point star plus the update
        flops, nbytes = 16 * per, (4 + 2 * w) * per
    elif name.startswith("stencil"):
        # flops per row: 13 for A x (7 multiply-adds less one), +1 for b - A x, +4 for the
        # Chebyshev update, +1 for x + d; bytes per row: the compulsory vector traffic
        # stencil_first alternates the step from x = 0 (2 flops; b in, d and x out) and the
        # step with c1 = 0 (17 flops; b, x in, d, x out): their mean
        flops = {"stencil_smooth": 19, "stencil_apply": 15, "stencil_resid": 14,
                 "stencil_first": 9.5}[name] * per
        nbytes = {"stencil_smooth": 5, "stencil_apply": 2, "stencil_resid": 3,
                  "stencil_first": 3.5}[name] * w * per
    else:
        # 2 flops per entry; bytes per entry: column index + value (FP32 / BF16 values in
        # the mixed V-cycle; transfers keep FP32 values in both mixed modes).  The level-1
        # smoother (coarse_csr) stores 16-bit column offsets when they fit (index_bytes 2).
        flops = 2 * per
        vbytes = 8 if prec == 0 else (2 if (prec == 2 and name.startswith("coarse")) else 4)
        ibytes = index_bytes if name == "coarse_csr" else 4
        nbytes = (ibytes + vbytes) * per
    out = {"kernel": name, "avg_launch_us": avg_s * 1e6, "launches": launches,
           "traffic": TRAFFIC_BYTES.get((name, prec, n)),
           "algorithmic_bytes_per_launch": nbytes, "algorithmic_flops_per_launch": flops}
    # FP64 stencil passes are bound by FP64 issue; the FP64 sparse passes move 12 B per
    # 2 flops, past the FP64 ridge of this part (1.26 TFLOP/s / 6.66 TB/s = 0.19 flop/B):
    # HBM is their tighter roofline, as for every FP32 / BF16 pass
    if prec == 0 and (name.startswith("stencil") or name == "prolong0"):
        ach = flops / avg_s / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": FP64_PEAK["tflops"], "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK["tflops"], "peak_source": FP64_PEAK["source"]})
    else:
        ach = nbytes / avg_s / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "peak_source": "measured" if peaks else "fallback"})
    return out


def level1_index_bytes(info):
    """Column bytes per stored entry of the level-1 smoother (SELL: 2 or 4; CSR: 4)."""
    ib = info.get("sell_index_bytes", [])
    return ib[1] if len(ib) > 1 and ib[1] else 4


def extra_legs(S, torch, w, dom, grid, rho, args):
    """Hierarchy reuse (Sec. 5.2, reusing the preconditioner) and the mixed-precision path."""
    out = {}
    for name, prec in (("fp64", 0), ("fp32", 1), ("bf16", 2)):
        params = S.params_default(max_coarse=4096, precision=prec, beta_rule=1 if prec else 0)
        op = shaped_operator(S, dom, grid, w.mode)
        h = S.setup(op, params)
        phi = torch.zeros_like(rho)
        S.solve(h, rho, phi, rtol=RTOL)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        its = []
        for k in range(args.steps):
            phi.zero_()
            its.append(S.solve(h, rho, phi, rtol=RTOL))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        # per-class kernel times on the host-driven loop (the same kernels, timed per launch)
        ht = S.setup(op, S.params_default(max_coarse=4096, precision=prec,
                                          beta_rule=1 if prec else 0, device_loop=0))
        S.solve(ht, rho, phi, rtol=RTOL)
        S.kernel_timing(True)
        for c in range(len(S.KT_NAMES)):
            S.kernel_timing_read(c)
        for k in range(args.steps):
            phi.zero_()
            S.solve(ht, rho, phi, rtol=RTOL)
        torch.cuda.synchronize()
        S.kernel_timing(False)
        kt = {S.KT_NAMES[c]: S.kernel_timing_read(c) for c in range(len(S.KT_NAMES))}
        ht.free()
        # whole pipeline in this precision
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            op2 = shaped_operator(S, dom, grid, w.mode)
            h2 = S.setup(op2, params)
            phi.zero_()
            S.solve(h2, rho, phi, rtol=RTOL)
            h2.free()
            op2.free()
        torch.cuda.synchronize()
        full_ms = 1e3 * (time.perf_counter() - t0) / args.steps
        out[f"{name}_vcycle"] = {
            "solve_only_solves_per_s": 1e3 / ms, "solve_ms": ms,
            "full_pipeline_solves_per_s": 1e3 / full_ms, "setup_ms": h.info()["setup_ms"],
            "iters": its[-1]["iters"], "relres_true": its[-1]["relres_true"],
            "rooflines": {c: roofline(c, kt[c], prec, args.n, level1_index_bytes(h.info()))
                          for c in SOLVE_CLASSES},
            "kernel_classes_ms_per_solve": {k: v[0] / args.steps for k, v in kt.items()},
            "solve_hbm": solve_hbm(h.info(), prec, its[-1]["iters"], ms),
        }
        h.free()
        op.free()
    # hierarchy reuse (Sec. 5.2): an operator with the same pattern (here the other boundary
    # mode on the same domain and grid) keeps the aggregates of an existing hierarchy
    params = S.params_default(max_coarse=4096)
    other = I.QUADRATIC if w.mode != I.QUADRATIC else I.LINEAR
    op1 = shaped_operator(S, dom, grid, w.mode)
    h1 = S.setup(op1, params)
    op2 = shaped_operator(S, dom, grid, other)
    S.setup_reuse(op2, h1, params).free()  # warm-up of both paths
    S.setup(op2, params).free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hf = S.setup(op2, params)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hr = S.setup_reuse(op2, h1, params)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    its = []
    for hh in (hf, hr):
        phi = torch.zeros_like(rho)
        its.append(S.solve(hh, rho, phi, rtol=RTOL)["iters"])
    out["hierarchy_reuse"] = {
        "operator": "same domain and grid, the other boundary mode (same pattern)",
        "fresh_setup_ms": 1e3 * (t1 - t0), "reuse_setup_ms": 1e3 * (t2 - t1),
        "iters_fresh": its[0], "iters_reuse": its[1]}
    for hh in (hf, hr, h1):
        hh.free()
    op1.free()
    op2.free()
    return out


def mixed_quadratic_leg(S, torch, args):
    """Quadratic extrapolation at 256^3 (mildly nonsymmetric): FP64 vs FP32 / BF16 V-cycle."""
    w = I.pipe_workload(args.n, I.QUADRATIC)
    dom, grid = S.make_domain(w.domain), S.make_grid(w.grid)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=77)).cuda()
    out, ref, sols = {}, None, {}
    for name, prec in (("fp64", 0), ("fp32", 1), ("bf16", 2)):
        params = S.params_default(max_coarse=4096, precision=prec, beta_rule=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = shaped_operator(S, dom, grid, w.mode)
        h = S.setup(op, params)
        phi = torch.zeros_like(rho)
        info = S.solve(h, rho, phi, rtol=RTOL)
        torch.cuda.synchronize()
        full = time.perf_counter() - t0
        ts = []
        for _ in range(3):
            phi2 = torch.zeros_like(rho)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            S.solve(h, rho, phi2, rtol=RTOL)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t1)
        if ref is None:
            ref = phi
        err = float((phi - ref).abs().max() / ref.abs().max())
        out[name] = {"full_pipeline_solves_per_s": 1.0 / full, "solve_only_solves_per_s": 1.0 / min(ts),
                     "iters": info["iters"], "relres_true": info["relres_true"],
                     "max_rel_diff_vs_fp64_gpu": err}
        sols[name] = phi.cpu().numpy()
        h.free()
        op.free()
    # error of every result against the FP64 oracle (multi-threaded build, same rhs): against
    # its solution at the same tolerance and against its rtol-1e-12 solution
    orc = oracle_solutions([{"workload": w, "seed": 77, "rtol": [1e-8, 1e-12], "beta_rule": 1}])
    if orc is not None:
        o8, o12 = orc["0_0"], orc["0_1"]
        for name, x in sols.items():
            out[name]["max_rel_err_vs_oracle"] = float(abs(x - o8).max() / abs(o8).max())
            out[name]["max_rel_err_vs_oracle_rtol_1e-12"] = float(abs(x - o12).max() / abs(o12).max())
    return {"mixed_quadratic_c3": {"workload": f"{w.name}, quadratic extrapolation, rtol 1e-8", **out}}


def vcycle_bytes(info, prec, degree=2):
    """Algorithmic bytes of one V-cycle from the level sizes: per smoothing or residual sweep
    the matrix entries (column + value) and the vectors; level 0 is matrix-free (20 B per row
    per Chebyshev step in FP32, 40 in FP64); transfers read P and R once each."""
    w = 8 if prec == 0 else 4
    n, nnz, nnz_p = info["n"], info["nnz"], info["nnz_p"]
    total = n[0] * w * (10 * degree + 3) + 2 * nnz_p[0] * (w + 4)
    for l in range(1, len(n) - 1):
        total += (2 * degree + 1) * nnz[l] * (w + 4) + n[l] * w * (10 * degree + 3)
        total += 2 * nnz_p[l] * (w + 4)
    total += n[-1] * n[-1] * 8  # explicit inverse of the coarsest operator
    return total


def solve_hbm(info, prec, iters, solve_ms, degree=2):
    """The whole solve against the HBM roofline: algorithmic bytes per PCG iteration (the
    FP64 CG vectors, 88 B per unknown: A p, the x / r update, p = z + beta p; plus one V-cycle)
    times the iterations, over the measured solve time."""
    per_iter = 88 * info["n"][0] + vcycle_bytes(info, prec, degree)
    gbs = per_iter * iters / (solve_ms * 1e-3) / 1e9
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(path)) if os.path.exists(path) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    return {"bytes_per_iteration": per_iter, "achieved_gbs": gbs, "peak_gbs": hbm,
            "frac": gbs / hbm, "peak_source": "measured" if peaks else "fallback"}


def aggregation_leg(S, torch, args):
    """MIS-2 aggregates against the paper's 3^3 cubes (Sec. 3.2) on the same workload:
    hierarchy, CG iterations, setup and solve time, V-cycle bytes."""
    w = workload(args.n)
    dom, grid = S.make_domain(w.domain), S.make_grid(w.grid)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=11)).cuda()
    out = {"workload": f"{w.name}, linear extrapolation, rtol 1e-8"}
    for name, agg in (("mis2", 0), ("cubes", 1)):
        for pname, prec in (("fp64", 0), ("fp32", 1)):
            params = S.params_default(max_coarse=4096, aggregation=agg, precision=prec,
                                      beta_rule=1 if prec else 0)
            op = shaped_operator(S, dom, grid, w.mode)
            h = S.setup(op, params)  # warm-up of this configuration
            h.free()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = S.setup(op, params)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            phi = torch.zeros_like(rho)
            info = S.solve(h, rho, phi, rtol=RTOL)
            phi.zero_()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            info = S.solve(h, rho, phi, rtol=RTOL)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            hi = h.info()
            out[f"{name}_{pname}"] = {
                "levels": hi["n"], "nnz": hi["nnz"], "iters": info["iters"],
                "relres_true": info["relres_true"], "setup_ms": 1e3 * (t1 - t0),
                "solve_ms": 1e3 * (t3 - t2), "vcycle_bytes": vcycle_bytes(hi, prec),
                "hierarchy_device_bytes": hi["device_bytes"]}
            h.free()
            op.free()
    return out


def coarse_solver_leg(S, torch, args):
    """Dense LU against three symmetric Gauss-Seidel steps on the coarsest level (Sec. 3.2):
    setup time, CG iterations and solve time on the same workload, both aggregations."""
    w = workload(args.n)
    dom, grid = S.make_domain(w.domain), S.make_grid(w.grid)
    rho = torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, seed=13)).cuda()
    out = {"workload": f"{w.name}, linear extrapolation, rtol 1e-8, FP64"}
    op = shaped_operator(S, dom, grid, w.mode)
    for aname, agg in (("mis2", 0), ("cubes", 1)):
        for cname, cs in (("lu", 0), ("gs3", 1)):
            params = S.params_default(max_coarse=4096, aggregation=agg, coarse_solver=cs)
            S.setup(op, params).free()  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = S.setup(op, params)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            phi = torch.zeros_like(rho)
            S.solve(h, rho, phi, rtol=RTOL)
            phi.zero_()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            info = S.solve(h, rho, phi, rtol=RTOL)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            out[f"{aname}_{cname}"] = {"coarse_n": h.info()["n"][-1], "iters": info["iters"],
                                       "relres_true": info["relres_true"],
                                       "setup_ms": 1e3 * (t1 - t0), "solve_ms": 1e3 * (t3 - t2)}
            h.free()
    op.free()
    return out


def pic_leg(S, torch, args, nparticles=10_000_000, reps=5):
    """The steps around the solve in a PIC time step (Sec. 1, Sec. 4.1) at the bench grid:
    CIC deposition of a Gaussian bunch of macro-particles, E = -grad phi, CIC gather.
    Times from CUDA events on the launching stream, inputs resident."""
    w = workload(args.n)
    G = S.make_grid(w.grid)
    op = S.build_operator(S.make_domain(w.domain), G, w.mode)
    x, y, z, q = (torch.from_numpy(a).cuda() for a in
                  I.bunch_particles(w.grid, nparticles, w.centre, w.sigma, seed=21))
    nbox = w.grid.nbox
    rho = torch.empty(nbox, dtype=torch.float64, device="cuda")
    e = [torch.empty(nbox, dtype=torch.float64, device="cuda") for _ in range(3)]
    ep = [torch.empty(nparticles, dtype=torch.float64, device="cuda") for _ in range(3)]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_dep = timed(lambda: S.deposit_cic(G, x, y, z, q, rho))
    phi = rho  # any box field: the gradient's cost does not depend on the values
    t_grad = timed(lambda: S.field_gradient(op, phi, *e))
    t_gat = timed(lambda: S.gather_cic(G, *e, x, y, z, *ep))
    op.free()
    return {"grid": list(w.grid.n), "particles": nparticles,
            "deposit_ms": t_dep, "deposit_particles_per_s": nparticles / (t_dep / 1e3),
            "gradient_ms": t_grad,
            "gradient_gbs": (nbox * 8 * 4) / (t_grad / 1e3) / 1e9,  # phi read, 3 fields written
            "gather_ms": t_gat, "gather_particles_per_s": nparticles / (t_gat / 1e3),
            "gather_gbs": (nparticles * 48) / (t_gat / 1e3) / 1e9}  # x, y, z in; 3 fields out


def sizes_leg(S, torch, sizes=(128, 256, 512)):
    """The elliptic-pipe workload at 128^3, 256^3 and 512^3 (linear, rtol 1e-8, coarse <= 4096):
    hierarchy, CG iterations (grid independence, Sec. 5), setup / solve / full-pipeline time,
    FP64 and the FP32 V-cycle.  One warm-up pass, then one timed pass per size."""
    out = {}
    for n in sizes:
        w = workload(n)
        dom, grid = S.make_domain(w.domain), S.make_grid(w.grid)
        rho = I.gaussian_bunch_torch(w.grid, w.centre, w.sigma, 31)
        for pname, prec in (("fp64", 0), ("fp32", 1)):
            params = S.params_default(max_coarse=4096, precision=prec, beta_rule=1 if prec else 0)
            for rep in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                op = shaped_operator(S, dom, grid, w.mode)
                h = S.setup(op, params)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                phi = torch.zeros_like(rho)
                info = S.solve(h, rho, phi, rtol=RTOL)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                hi = h.info()
                h.free()
                op.free()
            out[f"{n}^3_{pname}"] = {
                "unknowns": hi["n"][0], "levels": hi["n"], "iters": info["iters"],
                "sell_index_bytes": hi.get("sell_index_bytes"),
                "relres_true": info["relres_true"], "build_setup_ms": 1e3 * (t1 - t0),
                "solve_ms": 1e3 * (t2 - t1), "full_pipeline_solves_per_s": 1.0 / (t2 - t0)}
        del rho
        torch.cuda.empty_cache()
    return out


def batched_leg(S, torch):
    """64 instances of uneven grids (48..160 per axis) and geometries, 4 rhs each: one batched
    call with the FP32 V-cycle and autotuned Chebyshev degree, against FP64 solved one by one."""
    inst = I.batched_instances()
    hs32, hs64, rhos = [], [], []
    degrees = []
    # stencil launch shape per instance class (geometry kind, grid volume to a factor of 2),
    # tuned on the class's first instance and reused for the others
    shapes = {}
    for k, w in enumerate(inst):
        dom, grid = S.make_domain(w.domain), S.make_grid(w.grid)
        op = S.build_operator(dom, grid, w.mode)
        cls = (k % 3, int(math.log2(w.grid.nbox)))
        if cls not in shapes:
            shapes[cls] = S.autotune_stencil(op, 1)[0]
        S.set_stencil_config(op, 1, shapes[cls])
        h32 = S.setup(op, S.params_default(max_coarse=4096, precision=1, beta_rule=1))
        h64 = S.setup(op, S.params_default(max_coarse=4096))
        r = [torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 1234 + 4 * k + j)).cuda()
             for j in range(4)]
        best, _ = S.autotune_cheb_degree(h32, r[0], 2, 4)
        degrees.append(best)
        hs32.append(h32)
        hs64.append(h64)
        rhos.append(r)
    H = [h for h in hs32 for _ in range(4)]
    R = [r for rr in rhos for r in rr]
    X = [torch.zeros_like(r) for r in R]
    # the first call runs the merged form (one launch per operation across all solves), the
    # second the per-solve form (one device-loop graph per solve, concurrent branches); both
    # give the same bits, and later calls take the faster
    forms = {}
    for _ in range(2):
        for x in X:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.solve_batched(H, R, X)
        torch.cuda.synchronize()
        forms[S.batch_last()["form"]] = len(R) / (time.perf_counter() - t0)
    first = S.batch_last()
    for x in X:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = S.solve_batched(H, R, X)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t0
    chosen = S.batch_last()["form"]
    # FP32 one solve at a time (the same hierarchies and degrees)
    X1 = [torch.zeros_like(r) for r in R]
    S.solve(H[0], R[0], X1[0])
    X1[0].zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h, r, x in zip(H, R, X1):
        S.solve(h, r, x)
    torch.cuda.synchronize()
    t_seq32 = time.perf_counter() - t0
    same32 = all(bool(torch.equal(a, b)) for a, b in zip(X, X1))
    # FP64, one solve at a time through the synchronous call
    X64 = [torch.zeros_like(r) for r in R]
    H64 = [h for h in hs64 for _ in range(4)]
    S.solve(H64[0], R[0], X64[0])
    X64[0].zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its64 = [S.solve(h, r, x)["iters"] for h, r, x in zip(H64, R, X64)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    err = max(float((a - b).abs().max() / b.abs().max()) for a, b in zip(X, X64))
    # error against the FP64 oracle on a sample: every 8th instance, its 4 right-hand sides,
    # the oracle hierarchy with the instance's autotuned degree
    sample = list(range(0, len(inst), 8))
    cases = [{"workload": inst[k], "seed": 1234 + 4 * k + j, "rtol": [1e-8], "beta_rule": 1,
              "cheb_degree": degrees[k]} for k in sample for j in range(4)]
    orc = oracle_solutions(cases)
    err_orc = None
    if orc is not None:
        err_orc = {"fp32_batched": 0.0, "fp64_sequential": 0.0}
        for c, (k, j) in enumerate((k, j) for k in sample for j in range(4)):
            o = orc[f"{c}_0"]
            for key, xs in (("fp32_batched", X), ("fp64_sequential", X64)):
                x = xs[4 * k + j].cpu().numpy()
                err_orc[key] = max(err_orc[key], float(abs(x - o).max() / abs(o).max()))
    out = {"instances": len(inst), "solves": len(R),
           "unknowns_total": int(sum(h.info()["n"][0] for h in hs32) * 4),
           "batched_fp32_solves_per_s": len(R) / t_batched,
           "batched_form": chosen,
           "first_run_solves_per_s": {"merged": len(R) / (1e-3 * first["ms_merged"]) if first["ms_merged"] else None,
                                      "per_solve": len(R) / (1e-3 * first["ms_per_solve"]) if first["ms_per_solve"] else None},
           "sequential_fp32_solves_per_s": len(R) / t_seq32,
           "batched_equals_sequential_fp32_bitwise": same32,
           "sequential_fp64_solves_per_s": len(R) / t_seq,
           "speedup": t_seq / t_batched,
           "all_converged": all(i["converged"] == 1 for i in infos),
           "max_relres_true": max(i["relres_true"] for i in infos),
           "max_rel_diff_vs_fp64": err,
           "max_rel_err_vs_oracle": err_orc,
           "oracle_sample": f"instances {sample} x 4 rhs ({len(cases)} solves)",
           "autotuned_degrees": {d: degrees.count(d) for d in sorted(set(degrees))},
           "stencil_shape_classes": len(shapes),
           "iters_fp32_mean": statistics.fmean(i["iters"] for i in infos),
           "iters_fp64_mean": statistics.fmean(its64)}
    for h in hs32 + hs64:
        h.free()
    S.release_batch_cache()
    out["small_grids"] = batched_small_leg(S, torch)
    return out


def batched_small_leg(S, torch, count=64, lo=32, hi=48):
    """The same kind of batch on small grids (n_i ~ U{32..48}, 4 rhs each, FP32 V-cycle): the
    regime where a per-solve launch is mostly latency, so the merged form (one launch per
    operation across all solves) wins.  Both forms and one solve at a time."""
    inst = I.batched_instances(count=count, seed=5, lo=lo, hi=hi)
    H, R = [], []
    for k, w in enumerate(inst):
        op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
        h = S.setup(op, S.params_default(max_coarse=300, precision=1, beta_rule=1))
        h._op = op
        for j in range(4):
            H.append(h)
            R.append(torch.from_numpy(I.gaussian_bunch(w.grid, w.centre, w.sigma, 7 + 4 * k + j)).cuda())
    X = [torch.zeros_like(r) for r in R]
    rates = {}
    for _ in range(4):
        for x in X:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.solve_batched(H, R, X)
        torch.cuda.synchronize()
        form = S.batch_last()["form"]
        rates[form] = max(rates.get(form, 0.0), len(R) / (time.perf_counter() - t0))
    X1 = [torch.zeros_like(r) for r in R]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h, r, x in zip(H, R, X1):
        S.solve(h, r, x)
    torch.cuda.synchronize()
    seq = len(R) / (time.perf_counter() - t0)
    S.release_batch_cache()
    return {"instances": count, "solves": len(R), "grid_range": [lo, hi],
            "unknowns_total": int(sum(h.info()["n"][0] for h in H)),
            "merged_solves_per_s": rates.get("merged"), "per_solve_solves_per_s": rates.get("per-solve"),
            "sequential_fp32_solves_per_s": seq,
            "batched_equals_sequential_bitwise": all(bool(torch.equal(a, b)) for a, b in zip(X, X1))}


def serving_leg(S, torch, nreq):
    """The 10,000-request Poisson stream (mean gap 2 ms) over 20 geometries: the whole stream
    (or its first nreq requests) with FP32 continuous batching, then the same stream slowed
    to an offered load of about 0.8 of the throughput that replay measured (latency at a load
    the server sustains), and a prefix with warm starts and with FP64 one-at-a-time solves."""
    import dataclasses
    from paper_0907_4863_gb300 import serve
    geoms = I.serving_geometries()
    stream = I.serving_requests(10000)
    keys = ("solves_per_s", "offered_per_s", "p50_ms", "p99_ms", "mean_ms", "queue_p50_ms",
            "queue_p99_ms", "service_p50_ms", "service_p99_ms", "service_mean_ms", "wall_s",
            "cache_misses", "work_sets", "max_inflight_same_geometry", "all_converged", "rejected")
    fp32 = S.params_default(max_coarse=4096, precision=1, beta_rule=1)
    out = {"requests": 10000, "mean_gap_ms": 2.0, "geometries": len(geoms), "slots": 16,
           "work_sets_per_geometry": 4}

    def run(name, reqs, params, slots=16, warm=False, sets=4):
        srv = serve.Server(geoms, budget_bytes=120 << 30, slots=slots, params=params,
                           warm_start=warm, sets_per_geometry=sets)
        _, st = srv.run(reqs)
        srv.close()
        torch.cuda.synchronize()
        out[name] = {"requests_replayed": len(reqs), **{k: st[k] for k in keys}}
        return st

    full = run("fp32_continuous_batching", stream[:nreq], fp32)
    solo = solo_solve_ms(S, torch, geoms, fp32)
    out["fp32_solo_solve_ms"] = {geoms[g].name: round(v, 3) for g, v in solo.items()}
    busy_s = sum(solo[r.geometry] for r in stream[:nreq]) / 1e3
    out["fp32_one_after_another_solves_per_s"] = nreq / busy_s
    # the same arrivals stretched so that the offered rate is 0.8 x the measured throughput
    # (never faster than the stream itself)
    prefix = stream[:min(nreq, 3000)]
    mean_gap = prefix[-1].arrival / len(prefix)
    scale = max(1.0, 1.0 / (0.8 * full["solves_per_s"] * mean_gap))
    slowed = [dataclasses.replace(r, arrival=r.arrival * scale) for r in prefix]
    run("fp32_continuous_batching_load_0.8", slowed, fp32)
    short = stream[:min(nreq, 1500)]
    run("fp32_continuous_batching_warm_start", short, fp32, warm=True)
    run("fp64_one_at_a_time", short, S.params_default(max_coarse=4096), slots=1, sets=1)
    return out


def solo_solve_ms(S, torch, geoms, params):
    """Device time of one asynchronous solve (gather, device-loop graph, scatter) of each
    geometry's first time step, alone on the GPU (after a first solve that captures the
    graph): the requests' service times without any overlap."""
    out = {}
    st = torch.cuda.current_stream()
    for g, w in enumerate(geoms):
        op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode)
        h = S.setup(op, params)
        rho = I.gaussian_bunch_torch(w.grid, w.centre, w.sigma, 1000 * g)
        phi = torch.zeros_like(rho)
        S.solve_async(h, rho, phi, 1e-8, stream=st.cuda_stream)
        S.solve_wait(h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        phi.zero_()
        e0.record(st)
        S.solve_async(h, rho, phi, 1e-8, stream=st.cuda_stream)
        e1.record(st)
        S.solve_wait(h)
        e1.synchronize()
        out[g] = e0.elapsed_time(e1)
        h.free()
        op.free()
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm, errors against the oracle).  The oracle runs in a
# process of its own (python -m oracle.baseline): its OpenMP threads stay out of this one.
# ---------------------------------------------------------------------------
def oracle_process(extra, timeout=900):
    """Runs oracle/baseline.py with the given arguments; its JSON line, or None on failure."""
    cmd = [sys.executable, "-m", "oracle.baseline"] + [str(a) for a in extra]
    try:
        p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        print("oracle process timed out: " + " ".join(cmd), file=sys.stderr)
        return None
    if p.returncode != 0:
        print("oracle process failed: " + p.stderr[-2000:], file=sys.stderr)
        return None
    return json.loads(p.stdout.strip().splitlines()[-1])


def oracle_solutions(cases, timeout=900):
    """The FP64 oracle's solutions of the cases (see oracle.baseline.solve_cases), computed
    by its multi-threaded build on this host's cores; None if it is unavailable."""
    import tempfile
    import numpy as np
    from oracle.baseline import workload_to_dict
    with tempfile.TemporaryDirectory() as d:
        spec = os.path.join(d, "cases.json")
        out = os.path.join(d, "sol.npz")
        json.dump([{**c, "workload": workload_to_dict(c["workload"])} for c in cases], open(spec, "w"))
        if oracle_process(["--solve", spec, "--out", out, "--openmp"], timeout) is None:
            return None
        z = np.load(out)
        return {k: z[k] for k in z.files}


def cpu_baseline(n=256):
    """One full oracle pass (build + setup + PCG to rtol 1e-8) on the workload, OpenMP build
    on every core of the host, timed in its own process."""
    r = oracle_process(["--n", n, "--mode", "linear", "--passes", 1, "--openmp"])
    if r is None:
        return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                "sample": "the oracle process failed"}
    return {"value": r["solves_per_s"], "unit": UNIT, "cores": r["threads"], "kind": "oracle",
            "sample": f"one full FP64 oracle pass on {r['workload']} (build {r['build_s']:.2f} s + "
                      f"setup {r['setup_s']:.2f} s + PCG {r['solve_s']:.2f} s, {r['iters'][0]} "
                      f"iterations to rtol 1e-8), OpenMP build of the oracle on {r['threads']} threads",
            "build_s": r["build_s"], "setup_s": r["setup_s"], "solve_s": r["solve_s"]}


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper ships no code; the oracle is the one
    implementation of the method besides this library), OpenMP build on every host core,
    each step one full pass of the workload: build + setup + PCG to rtol 1e-8, measured."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    r = oracle_process(["--n", args.n, "--mode", "linear", "--passes", args.steps,
                        "--warmup", args.warmup, "--openmp"], timeout=3600)
    if r is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle process failed"}), flush=True)
        return
    value = r["solves_per_s"]
    w = workload(args.n)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["total_s"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Gaussian bunch, no dataset)",
           "config": {"workload": f"{w.name}, linear extrapolation, Robin ends, rtol 1e-8, coarse <= 4096; "
                                  "step = build operator + AMG setup + PCG solve",
                      "grid": list(w.grid.n), "parallelism": f"CPU, {r['threads']} OpenMP threads"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["threads"], "kind": "oracle",
                            "sample": f"each step one full FP64 oracle pass (build + setup + PCG to rtol 1e-8), "
                                      f"OpenMP build on {r['threads']} of {r['host_cores']} host cores"},
           "phases_s": {k: r[k] for k in ("build_s", "setup_s", "solve_s")}, "iters": r["iters"],
           "relres_true_max": r["relres_true_max"],
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_leg(args):
    """One extra leg on its own (for profiling it or running it alone)."""
    import torch
    from paper_0907_4863_gb300 import saamg as S
    _, local, _ = dist_env()
    torch.cuda.set_device(local)
    S.use_torch_allocator()
    if args.leg == "batched":
        out = batched_leg(S, torch)
    else:
        out = serving_leg(S, torch, args.serve_requests)
    print(json.dumps({"leg": args.leg, **out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.leg:
        run_leg(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
