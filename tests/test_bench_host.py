"""Host-side pieces of bench.py: the roofline arithmetic of each timing class."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fp64_stencil_is_reported_against_the_fp64_issue_peak(bench):
    # 10 launches of 1e6 rows, 100 us each: 19 flops per row -> 0.19 TFLOP/s
    r = bench.roofline("stencil_smooth", (1.0, 10, 10_000_000), 0, n=128)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(0.19)
    assert r["frac"] == pytest.approx(0.19 / bench.FP64_PEAK["tflops"])
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(40e6)
    assert r["traffic"] is None  # no capture for this size


def test_fp32_stencil_and_sparse_classes_are_reported_against_hbm(bench):
    r = bench.roofline("stencil_smooth", (1.0, 10, 10_000_000), 1)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(20e6 / 100e-6 / 1e9)
    # sparse classes count matrix entries: 8 bytes per entry in FP32, 6 with BF16 values
    r = bench.roofline("coarse_csr", (1.0, 10, 10_000_000), 1)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(8e6)
    r = bench.roofline("coarse_csr", (1.0, 10, 10_000_000), 2)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(6e6)
    r = bench.roofline("transfer", (1.0, 10, 10_000_000), 2)  # transfers keep FP32 values
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(8e6)
    # FP64 sparse passes sit past the FP64 ridge: reported against HBM, 12 B per entry
    r = bench.roofline("coarse_csr", (1.0, 10, 10_000_000), 0)
    assert r["bound"] == "hbm" and r["algorithmic_bytes_per_launch"] == pytest.approx(12e6)
    assert r["algorithmic_flops_per_launch"] == pytest.approx(2e6)
    # the CG product is FP64 in every precision mode
    assert bench.roofline("stencil_apply", (1.0, 10, 10_000_000), 1)["bound"] == "alu"


def test_empty_class_has_no_roofline(bench):
    assert bench.roofline("transfer", (0.0, 0, 0), 0) is None


def _replica(rank, world, port, local_seconds, out):
    import importlib.util
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    t = b.max_over_ranks(local_seconds[rank], world, "cpu")
    out[rank] = (t, b.whole_job_rate(world, 5, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_report_the_slowest_rank_over_gloo():
    """Two gloo ranks on the CPU: every rank gets the maximum of the local times, and the
    whole-job rate counts the solves of all replicas over that time."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        port = s_.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    local = [0.8, 1.25]
    ps = [ctx.Process(target=_replica, args=(r, 2, port, local, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r][0] == 1.25 and out[r][1] == pytest.approx(2 * 5 / 1.25)


def test_solve_hbm_counts_cg_vectors_and_one_vcycle_per_iteration(bench):
    info = {"n": [1000, 100, 10], "nnz": [7000, 2000, 60], "nnz_p": [3000, 300, 0]}
    # FP64, degree 2: level 0 1000*8*23 + 2*3000*12; level 1 5*2000*12 + 100*8*23 + 2*300*12;
    # coarsest 10^2 * 8; CG vectors 88 * 1000
    vc = 184000 + 72000 + 120000 + 18400 + 7200 + 800
    assert bench.vcycle_bytes(info, 0) == vc
    r = bench.solve_hbm(info, 0, iters=10, solve_ms=2.0)
    assert r["bytes_per_iteration"] == 88000 + vc
    assert r["achieved_gbs"] == pytest.approx((88000 + vc) * 10 / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved_gbs"] / r["peak_gbs"])


def test_level1_smoother_counts_its_column_bytes(bench):
    # 16-bit column offsets: 2 + 4 B per entry in FP32, 2 + 8 in FP64; transfers keep 4-byte columns
    assert bench.roofline("coarse_csr", (1.0, 10, 10_000_000), 1, index_bytes=2)[
        "algorithmic_bytes_per_launch"] == pytest.approx(6e6)
    assert bench.roofline("coarse_csr", (1.0, 10, 10_000_000), 0, index_bytes=2)[
        "algorithmic_bytes_per_launch"] == pytest.approx(10e6)
    assert bench.roofline("transfer", (1.0, 10, 10_000_000), 1, index_bytes=2)[
        "algorithmic_bytes_per_launch"] == pytest.approx(8e6)
    assert bench.level1_index_bytes({"sell_index_bytes": [0, 2, 0]}) == 2
    assert bench.level1_index_bytes({"sell_index_bytes": [0, 0, 0]}) == 4


def test_captured_traffic_is_attached_to_the_256_cube_classes(bench):
    """The ncu DRAM bytes per launch go with the class, precision and size they were captured
    on (the BF16 mode's level-0 passes are the FP32 kernels); nothing else carries any, and each
    capture stays near the class's algorithmic bytes at 7,119,872 rows."""
    rows = 7_119_872
    rec = (1.0, 10, 10 * rows)
    r = bench.roofline("stencil_smooth", rec, 0, n=256)
    assert r["traffic"] == pytest.approx(364.0e6)
    assert 1.0 < r["traffic"] / r["algorithmic_bytes_per_launch"] < 1.3  # the (row, line) list
    for prec in (1, 2):
        for name in ("stencil_smooth", "stencil_resid", "prolong0"):
            r = bench.roofline(name, rec, prec, n=256)
            assert r["traffic"] is not None
            assert 0.8 < r["traffic"] / r["algorithmic_bytes_per_launch"] < 1.1
        for name in ("stencil_first", "coarse_csr", "transfer", "coarse_deep"):
            assert bench.roofline(name, rec, prec, n=256)["traffic"] is None
    assert bench.roofline("stencil_resid", rec, 0, n=256)["traffic"] is None
    assert bench.roofline("stencil_smooth", rec, 1, n=512)["traffic"] is None
