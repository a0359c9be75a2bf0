"""The benchmark's roofline object on CPU: which kernel class it reports, the bound it picks
(arithmetic intensity against the ridge point of the two peaks), the achieved rate from the
accumulated bytes and operations over the event time, and the DRAM traffic it attaches from
the committed captures (per box cell for the Schwarz kernels; for residual pass A the mix of
its two captured forms over the timed launches)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads import PREC_FP64, PREC_MIXED  # noqa: E402

HBM = (6800.0, "test")
CELLS = 4194304


def test_alu_bound_class_and_pass_a_traffic_mix():
    # residual pass A dominates: 150 launches (50 first evaluations, 100 trial evaluations)
    n = 150
    flops = (50 * 114.0 + 100 * 226.0) * CELLS
    stats = {"residual_g": (n, 131.4, 330e6 * n, flops), "ras_apply": (200, 78.0, 1e9, 1e9)}
    r = bench.roofline(stats, PREC_MIXED, HBM, 1.25, None, None, None, CELLS, 50)
    assert r["kernel"] == "residual_g" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / (131.4e-3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.25)
    first, trial = bench.TRAFFIC_PASS_A[PREC_MIXED]
    assert r["traffic"] == pytest.approx(CELLS * (50 * first + 100 * trial) / n)
    # without the count of first evaluations no traffic is claimed
    assert bench.roofline(stats, PREC_MIXED, HBM, 1.25, None, None, None, CELLS)["traffic"] is None
    # the FP64 form has no capture of both forms: no traffic
    assert bench.roofline(stats, PREC_FP64, HBM, 1.25, None, None, None, CELLS, 50)["traffic"] is None


def test_box_kernel_traffic_and_hbm_bound():
    # the float apply dominates with few operations per byte: HBM bound, traffic per box cell
    box_cells = 4_481_956
    stats = {"ras_apply": (4, 1.56, 216.0 * box_cells * 4, 104.0 * box_cells * 4), "jvp_f": (4, 0.2, 1e8, 1e8)}
    r = bench.roofline(stats, PREC_MIXED, HBM, 1.25, box_cells, 124, None, CELLS)
    assert r["kernel"] == "ras_apply" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(216.0 * box_cells * 4 / 1.56e-3 / 1e9)
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_BOX_CELL[("ras_apply", PREC_MIXED, 124)] * box_cells)
    # a box width without a capture gets no traffic
    assert bench.roofline(stats, PREC_MIXED, HBM, 1.25, box_cells, 68, None, CELLS)["traffic"] is None


def test_share_of_kernel_time():
    stats = {"ras_factor": (1, 3.0, 1e9, 2.4e9), "ras_apply": (4, 1.0, 1e9, 1e9)}
    warm = {"ras_factor": (1, 3.0, 1e9, 2.4e9), "ras_apply": (4, 3.0, 1e9, 1e9), "residual_g": (3, 4.0, 1e9, 1e9)}
    r = bench.roofline(stats, PREC_FP64, HBM, 1.25, None, None, warm, CELLS)
    assert r["kernel"] == "ras_factor"
    assert r["share_of_kernel_time"] == pytest.approx(3.0 / 10.0)
