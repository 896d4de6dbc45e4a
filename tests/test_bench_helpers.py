"""Host logic of bench.py that decides the reported numbers: the algorithmic work per launch of the
roofline kernel (whole-Delta steps, multipole chunks, Delta recomputed in the VJP), the peak it is
divided by, and when a stored DRAM-traffic figure applies.  No GPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6777.3, "bf16_tflops": 1890.6, "bf16_tflops_sustained": 1739.2}


@pytest.fixture(scope="module")
def n5k():
    return bench.make_inputs(1, 0, 1)[0]


def test_contraction_count_matches_its_definition(n5k):
    # the real part of sum_n over n_h complex products for each (i, l, q): two multiply-adds,
    # 4 flops, per term
    work = bench.algorithmic_work(n5k, 1, 1)
    assert work["basis gemm adj"][1] == 4.0 * 1025 * 15 * 1024 * 103
    assert work["basis gemm adj"][2] == 6
    assert work["basis gemm fwd"][0] == "tensor"
    assert work["fftlog"][0] == "alu"


def test_roofline_of_a_whole_delta_step(n5k):
    flops = 4.0 * 1025 * 15 * 1024 * 103
    stats = {"basis gemm adj": (200, 200 * 0.0744), "basis gemm fwd": (200, 200 * 0.057)}
    r = bench.roofline(stats, n5k, 1, "bf16x9", PEAKS, "measured", 1, "n5k", 200, False)
    assert r["kernel"] == "basis gemm adj"
    # achieved and frac count the method's useful flops; the executed compensated products
    # (6 per useful multiply-add in basis mode) only enter the pipe occupancy
    assert r["achieved"] == pytest.approx(flops / 0.0744e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1890.6)
    assert r["pipe_occupancy"] == pytest.approx(6 * r["frac"])


def test_roofline_follows_chunks_and_recompute(n5k):
    flops = 4.0 * 1025 * 15 * 1024 * 103
    # three chunks per pass: the forward GEMM runs 3 + 3 (recompute) launches per step
    stats = {"basis gemm fwd": (30, 30 * 0.02), "basis gemm adj": (15, 15 * 0.025)}
    r = bench.roofline(stats, n5k, 1, "bf16x9", PEAKS, "measured", 1, "n5k", 5, True)
    assert r["kernel"] == "basis gemm fwd"
    assert r["achieved"] == pytest.approx(flops * 2 / 6 / 0.02e-3 / 1e12)
    # without recompute the same launches would be six chunks of one pass
    r2 = bench.roofline(stats, n5k, 1, "bf16x9", PEAKS, "measured", 1, "n5k", 5, False)
    assert r2["achieved"] == pytest.approx(r["achieved"] / 2)


def test_tf32_and_fp64_peaks(n5k):
    stats = {"contract tc": (10, 10 * 0.1)}
    # without a TF32 rate measured in the run: the bf16 peak times the nominal ratio
    r = bench.roofline(stats, n5k, 1, "tf32x6", PEAKS, "measured", 0, "n5k", 10)
    assert r["peak"] == pytest.approx(1890.6 * 1.1 / 2.25)
    assert r["products"] == 6
    measured = dict(PEAKS, tf32_tflops=950.0, fp64_tflops=1.1)
    r = bench.roofline(stats, n5k, 1, "tf32x6", measured, "measured", 0, "n5k", 10)
    assert r["peak"] == 950.0
    stats = {"contract fp64": (10, 10 * 5.0)}
    r = bench.roofline(stats, n5k, 1, "fp64", PEAKS, "measured", 0, "n5k", 10)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    r = bench.roofline(stats, n5k, 1, "fp64", measured, "measured", 0, "n5k", 10)
    assert r["peak"] == 1.1 and r["frac"] == pytest.approx(r["achieved"] / 1.1)


def test_ragged_lists_count_only_listed_multipoles(n5k):
    stats = {"basis gemm adj": (1, 1.0)}
    full = bench.roofline(stats, n5k, 2, "bf16x9", PEAKS, "measured", 1, "walkers", 1)
    part = bench.roofline(stats, n5k, 2, "bf16x9", PEAKS, "measured", 1, "walkers", 1,
                          n_ell_useful=103)
    assert part["achieved"] == pytest.approx(full["achieved"] / 2)


def test_named_kernel_roofline(n5k):
    stats = {"contract tc": (10, 1.0), "contract adj tc": (10, 2.0)}
    r = bench.roofline(stats, n5k, 1, "bf16x9", PEAKS, "measured", 0, "n5k", 10, kernel="contract tc")
    assert r["kernel"] == "contract tc" and r["products"] == 9
    assert bench.roofline(stats, n5k, 1, "bf16x9", PEAKS, "m", 0, "n5k", 10, kernel="nope") is None


def test_stored_traffic_applies_only_to_its_workload_source_and_tiles():
    t = bench.TRAFFIC[("basis gemm adj", 16608)]
    tiles = {"fwd": 1120, "adj": 16608}
    got = bench.traffic_for("basis gemm adj", 1, "n5k", tiles)
    assert got in (t["bytes"], None)     # None once the kernel source has changed
    assert bench.traffic_for("basis gemm adj", 1, "n5k") is None                       # tiles unknown
    assert bench.traffic_for("basis gemm adj", 1, "n5k", {"fwd": 1120, "adj": 96}) is None
    assert bench.traffic_for("basis gemm adj", 1, "large", tiles) is None
    assert bench.traffic_for("basis gemm adj", 256, "n5k", tiles) is None
    assert bench.traffic_for("fftlog", 1, "n5k", tiles) is None
