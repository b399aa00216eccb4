"""Host logic of bench.py's roofline: algorithmic work per kernel group, the bound
each group reports against, and the choice of the dominant (longest) kernel."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

COUNTS = {"exposures": 1000, "kept": 100, "in_window": 99, "kepler": 99, "items": 1500,
          "item_kepler": 0, "full": 600, "partial": 200}


def test_window_kernel_is_reported_against_the_copy_bandwidth():
    # 1000 exposures on a shared grid of 500 times: 4000 B of times, 900 fluxes of
    # 8 B written, 100 kept-list entries of 8 B
    assert bench.window_bytes(COUNTS, 8 * 500) == 4000 + 7200 + 800
    kern = {"window": 1e-3, "exposures": 0.5e-3, "quadrature": 0.2e-3}
    line = bench.roofline(COUNTS, kern, 77.0, 1.2, 6479.6, 8 * 500, "some_batch")
    assert line["bound"] == "hbm" and line["unit"] == "GB/s"
    assert line["kernel"] == "gl_win_kernel"
    assert abs(line["achieved"] - 12000 / 1e-6 / 1e9) < 1e-9
    assert abs(line["frac"] - line["achieved"] / 6479.6) < 1e-12
    assert line["traffic"] is None   # no capture for this workload
    assert set(line["kernels"]) == {"gl_win_kernel", "gl_expgeo_kernel",
                                    "gl_items_quad_kernel+gl_items_sum_kernel"}


def test_alu_groups_count_flops_per_unit_and_pick_the_binding_pipe():
    f = bench.kernel_flops(COUNTS)
    assert f["exposures"] == (1500 * bench.F32_ITEM,
                              100 * bench.F64_WINDOW + 99 * bench.F64_KEPLER)
    assert f["quadrature"] == (600 * bench.F32_FULL + 200 * bench.F32_PARTIAL,
                               200 * bench.F64_PARTIAL + 1500 * bench.F64_SUM)
    kern = {"window": 0.1e-3, "exposures": 0.2e-3, "quadrature": 1e-3}
    line = bench.roofline(COUNTS, kern, 77.0, 1.2, 6479.6, 8000, "mcmc_batch")
    assert line["kernel"] == "gl_items_quad_kernel+gl_items_sum_kernel"
    assert line["bound"] == "alu"
    f32, f64 = f["quadrature"]
    # the pipe with the larger share of its peak is the one reported
    want = "fp64" if f64 / 1.2 >= f32 / 77.0 else "fp32"
    assert line["pipe"] == want
    assert line["traffic"] == bench.TRAFFIC.get(("mcmc_batch", "quadrature"))


def test_missing_peaks_file_falls_back_and_says_so():
    r = bench.hbm_roofline(6.4e9, 1000.0, None)
    assert r["peak"] == 6400.0 and "fallback" in r["peak_source"]
    assert abs(r["frac"] - 1e-3) < 1e-12
