"""The ``roofline`` object of the bench line, on the CPU with synthetic stage figures: the
dominant stage is the slowest one, its bound is whichever of the modelled HBM and FP32 times
is larger, ``achieved`` is the algorithmic amount per launch over the measured stage time,
``frac`` is achieved over that bound's peak, and ``traffic`` is the committed capture of
that stage's kernel (or null)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KEYS = {"bound", "kernel", "achieved", "peak", "unit", "frac", "traffic", "peak_source",
        "alg_bytes", "alg_flops", "hbm_frac", "alu_frac", "stage_ms"}


def _stage(ms_by_stage, steps):
    # total milliseconds and launch count per stage, as bench.py accumulates them
    return {k: (v * steps, steps) for k, v in ms_by_stage.items()}


def test_alu_bound_dominant_stage():
    import bench
    steps = 4
    stage = _stage({"project": 0.02, "bin": 0.05, "fwd": 0.07, "bwd_raster": 0.18,
                    "bwd_project": 0.02}, steps)
    # 2 GFLOP and 50 MB per backward launch: 25 us at the FP32 peak against 7 us at HBM
    sb = {k: 1e6 * steps for k in stage}
    sb["bwd_raster"] = 50e6 * steps
    sf = {k: 1e6 * steps for k in stage}
    sf["bwd_raster"] = 2e9 * steps
    r = bench.build_roofline(stage, sb, sf, (1000 * steps, 100 * steps), steps,
                             "slam_640x480_200k")
    assert KEYS <= set(r)
    assert r["kernel"] == "bwd_raster" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    peak = bench.fp32_peak_tflops(bench.load_peaks()[0])
    assert r["achieved"] == pytest.approx(2e9 / 0.18e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-3)
    assert r["peak"] == pytest.approx(peak, abs=0.1)
    assert r["hbm_frac"] < r["alu_frac"]
    # the committed capture of this kernel on this workload, while its sources match
    assert r["traffic"] == bench.captured_traffic("bwd_raster", "slam_640x480_200k")
    assert r["pairs_eval_per_step"] == 1000 and r["pairs_blend_per_step"] == 100


def test_hbm_bound_dominant_stage_and_missing_capture():
    import bench
    steps = 2
    # the grid forward's shape: 560 MB and 3 GFLOP per launch (83 us at HBM, 37 us at FP32)
    stage = _stage({"fwd": 0.40, "bwd_raster": 0.39, "bin": 0.17}, steps)
    sb = {"fwd": 560e6 * steps, "bwd_raster": 570e6 * steps, "bin": 99e6 * steps}
    sf = {"fwd": 3e9 * steps, "bwd_raster": 2.9e9 * steps, "bin": 0.0}
    r = bench.build_roofline(stage, sb, sf, (0, 0), steps, "no_such_workload")
    peaks, src = bench.load_peaks()
    assert r["kernel"] == "fwd" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(560e6 / 0.40e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peaks["hbm_gbs"], rel=1e-3)
    assert r["peak_source"] == src
    assert r["traffic"] is None   # no capture recorded for this workload


def test_measured_fp32_peak_is_the_alu_denominator():
    import bench
    steps = 3
    stage = _stage({"fwd": 0.07, "bwd_raster": 0.18, "bin": 0.05}, steps)
    sb = {"fwd": 40e6 * steps, "bwd_raster": 50e6 * steps, "bin": 6e6 * steps}
    sf = {"fwd": 0.8e9 * steps, "bwd_raster": 2e9 * steps, "bin": 0.0}
    fp32 = {"tflops": 70.0, "sm_mhz": 1900.0}
    r = bench.build_roofline(stage, sb, sf, (0, 0), steps, "no_such_workload", fp32, 2000.0)
    achieved = 2e9 / 0.18e-3 / 1e12
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(70.0)
    assert r["peak_source"].startswith("measured")
    assert r["frac"] == pytest.approx(achieved / 70.0, rel=1e-3)
    assert r["alu_frac"] == pytest.approx(achieved / 70.0, rel=1e-3)
    # the same fraction against the peak scaled to the clock the kernel ran at
    assert r["alu_frac_at_kernel_clock"] == pytest.approx(achieved / (70.0 * 2000 / 1900), rel=1e-3)
    assert r["stage_kcycles"] == pytest.approx(0.18 * 2000.0, rel=1e-3)
