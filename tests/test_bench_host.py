"""Host-side arithmetic of bench.py (no GPU): the per-kernel roofline
fractions and the FLOP model they use."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_rooflines_divide_algorithmic_work_by_time_and_peak():
    kms = {"project": 0.1, "depth_sort": 0.05, "tile_scan": 0.02, "emit": 0.08, "tile_sort": 0.16, "ranges": 0.03,
           "raster_fwd": 0.5, "raster_bwd": 1.0, "project_bwd": 0.07, "adam": 0.025}
    N, M, P, T = 200_000, 1_600_000, 10_000_000, 10_240
    n_params = N * 23
    out = bench.kernel_rooflines(kms, N, M, P, T, n_params, 92, 0, visited=5e8, contrib=2e8, ffma_tflops=75.0,
                                 hbm_gbs=6500.0)
    assert set(out) == set(kms)
    # HBM-bound kernels: bytes per unit x units / time / measured copy rate
    assert out["tile_sort"]["work"] == P * 16.0
    assert out["tile_sort"]["achieved"] == pytest.approx(P * 16.0 / 0.16e-3 / 1e9)
    assert out["adam"]["work"] == n_params * 28.0
    assert out["adam"]["frac"] == pytest.approx(n_params * 28.0 / 0.025e-3 / 1e9 / 6500.0)
    assert out["project"]["work"] == M * (92 + 80.0)
    # compositing: the FLOP model, 12 per visited fragment plus 10 (forward) or 34 (backward) per contributing one
    assert out["raster_bwd"]["bound"] == "alu"
    assert out["raster_bwd"]["work"] == pytest.approx(12 * 5e8 + 34 * 2e8)
    assert out["raster_fwd"]["work"] == pytest.approx(12 * 5e8 + 9 * 2e8)
    assert out["raster_bwd"]["frac"] == pytest.approx((12 * 5e8 + 34 * 2e8) / 1e-3 / 1e12 / 75.0)
    # a kernel that did not run is left out
    out2 = bench.kernel_rooflines({"adam": 0.02}, N, M, P, T, n_params, 92, 0, 0, 0, 75.0, 6500.0)
    assert list(out2) == ["adam"]


def test_low_precision_copy_adds_its_bytes():
    a = bench.kernel_rooflines({"adam": 0.02}, 10, 10, 10, 1, 230, 52, 0, 0, 0, 75.0, 6500.0)["adam"]["work"]
    b = bench.kernel_rooflines({"adam": 0.02}, 10, 10, 10, 1, 230, 52, 200, 0, 0, 75.0, 6500.0)["adam"]["work"]
    assert b - a == 200 * 2.0


def test_split_bins_count_their_pairs_lists_and_tiles():
    """Bins of several tiles: the ranges count bins, the split reads each
    (bin, record) pair's key and record and writes every list entry and
    tile range."""
    P, Tb, T, n_list = 4_873_213, 2560, 40_960, 29_290_925
    out = bench.kernel_rooflines({"ranges": 0.03, "refine": 0.06}, 200_000, 1_600_000, P, T, 4_600_000, 92, 0,
                                 0, 0, 75.0, 6500.0, n_bins=Tb, n_list=n_list)
    assert out["ranges"]["work"] == P * 4.0 + Tb * 8.0
    assert out["refine"]["work"] == P * 8.0 + n_list * 4.0 + T * 8.0
    assert out["refine"]["frac"] == pytest.approx((P * 8.0 + n_list * 4.0 + T * 8.0) / 0.06e-3 / 1e9 / 6500.0)
