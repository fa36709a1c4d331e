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
    assert r["frac"] == pytest.approx(0.19 / bench.FP64_PEAK_TFLOPS)
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
