"""The roofline arithmetic of bench.py (CPU): the algorithmic work per stage launch that the bench
line divides by each stage's CUDA-event time.  The expected figures are written out from the plan
of the benchmark's workload (spin 2, lmax 4096, eps 1e-5: L = 960 rings, M = 2659, 1759 kept rows,
n_phi = 10752, 2.23e7 points, 4.33e9 recursion triples), so a changed byte or flop count fails."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

INFO = dict(M=2659, nring=960, nrows=1759, nphi=10752, npts=22_322_966, W=6, recursion_triples=4_332_618_634)
MS = dict(rec_synthesis=2.0, theta_synthesis=0.3, phi_synthesis=0.2, gather=0.3,
          scatter=0.75, phi_adjoint=0.2, theta_adjoint=0.3, rec_adjoint=2.5)


def test_flops_per_triple():
    # two Wigner columns for s > 0 (3-term step of 2 FMA and complex-by-real accumulation of 2 FMA
    # each: 8 FMA = 16 flops); one column for s = 0 plus the two complex accumulations (12 flops)
    assert bench.flops_per_triple(2) == 16
    assert bench.flops_per_triple(1) == 16
    assert bench.flops_per_triple(0) == 12


def test_stage_work_of_the_benchmark_plan():
    r = bench.stage_rooflines(INFO, MS, "fp32", 2)
    assert set(r) == set(MS)
    assert r["rec_synthesis"]["flops"] == 4_332_618_634 * 16 == r["rec_adjoint"]["flops"]
    # Theta stages: ring coefficients (960 x 5319) and kept rows (1759 x 5319), complex64
    assert r["theta_synthesis"]["bytes"] == (960 + 1759) * 5319 * 8 == 115_698_888
    # phi stages: kept rows (1759 x 5319) and grid rows (1759 x 10752)
    assert r["phi_adjoint"]["bytes"] == 1759 * (5319 + 10752) * 8 == 226_151_112
    # interpolation: 16 B of coordinates and one complex64 value per point, plus the grid rows
    assert r["gather"]["bytes"] == 22_322_966 * 24 + 1759 * 10752 * 8 == r["scatter"]["bytes"]
    for st, e in r.items():
        per_s = (e["flops"] / 1e12 if e["bound"] == "alu" else e["bytes"] / 1e9) / (MS[st] * 1e-3)
        assert e["achieved"] == pytest.approx(per_s, rel=1e-12)
        assert e["frac"] == pytest.approx(e["achieved"] / e["peak"], rel=1e-12)
        assert e["kernel"] == bench.STAGE_KERNELS[st]["fp32"]
    assert r["scatter"]["kernel"] == "k_scatter_rows" and r["rec_adjoint"]["kernel"] == "k_rec_adj_w"


def test_peaks_fp32_lanes_and_fp64_rate():
    # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz; FP64 at 1/64 of it
    assert bench.alu_peak_tflops(32) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12, rel=1e-12)
    assert bench.alu_peak_tflops(64) == pytest.approx(bench.alu_peak_tflops(32) / 64, rel=1e-12)
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        gbs, note = bench.hbm_peak()
        assert "measured" in note and gbs > 1000


def test_fp64_interpolation_also_carries_its_fp64_flops():
    info = dict(INFO, W=11)
    r = bench.stage_rooflines(info, MS, "fp64", 2)
    assert r["gather"]["bytes"] == 22_322_966 * 32 + 1759 * 10752 * 16
    assert r["gather"]["alu"]["flops"] == (4 * 121 + 4 * 11) * 22_322_966
    assert r["scatter"]["alu"]["flops"] == (4 * 121 + 2 * 11) * 22_322_966
    assert r["scatter"]["kernel"] == "k_scatter"


def test_kernel_traffic_names_known_stages():
    for (form, stage), v in bench.KERNEL_TRAFFIC.items():
        assert form in ("fp32", "fp64") and stage in bench.STAGE_KERNELS
        assert v is None or v > 1e8
