"""Host-side arithmetic of bench.py's per-phase rooflines (no GPU): FP64-pipe
phases are rated in TFLOP/s against the derived FP64 peak, memory-bound phases
in GB/s against the measured copy bandwidth, time-only phases carry no rate."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_phase_rooflines():
    prof = {"apply": (2.0e12, 2000.0, 4), "precond": (6.0e9, 2.0, 4), "factor": (0.0, 30.0, 1),
            "recover": (0.0, 3.0, 1), "project": (0.0, 0.0, 0), "gram": (1.0e12, 1000.0, 8),
            "step": (1.0e9, 1.0, 8), "ortho": (0.0, 5.0, 4)}
    out = bench.phase_rooflines(prof, steps=2, t_steps=4.0)
    a = out["apply"]
    assert a["ms_per_step"] == pytest.approx(1000.0)
    assert a["share_of_step"] == pytest.approx(0.5)
    assert a["bound"] == "alu" and a["unit"] == "TFLOP/s"
    assert a["achieved"] == pytest.approx(1.0)
    assert a["frac"] == pytest.approx(1.0 / bench.FP64_PEAK_TFLOPS)
    p = out["precond"]
    assert p["bound"] == "hbm" and p["unit"] == "GB/s"
    assert p["achieved"] == pytest.approx(3000.0)
    assert p["frac"] == pytest.approx(3000.0 / bench.tensor_peaks()["hbm_gbs"])
    assert "achieved" not in out["factor"] and "achieved" not in out["ortho"]   # no work recorded
    assert "project" not in out                                                 # never entered
