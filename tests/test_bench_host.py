"""Host-side arithmetic of bench.py's rooflines (no GPU): per phase, FP64-pipe
phases are rated in TFLOP/s against the derived FP64 peak, memory-bound phases
in GB/s against the measured copy bandwidth, time-only phases carry no rate;
for the tensor-core products the binding limit of max(bytes / HBM bandwidth,
passes x flops / tensor peak) is reported."""
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


class _FakeLib:
    """Stands in for the binding: a profile of 2 launches of 1 ms, fixed byte counts."""
    FETI_TF32, FETI_TF32X3, FETI_BF16, FETI_BF16X3 = 1, 2, 3, 4
    FETI_Q_TC_BYTES_F, FETI_Q_TC_BYTES_PER_COL = 13, 14

    def __init__(self, flops):
        self.flops = flops

    def feti_profile_tensor(self, ctx):
        return 2 * self.flops, 2.0, 2

    def feti_query(self, ctx, key):
        return {13: 2_000_000_000, 14: 4_000_000}[key]


class _S:
    ctx = None


def test_tensor_roofline_picks_the_binding_limit():
    pk = bench.tensor_peaks()
    # one BF16 pass: 2.0 GB + 512 x 4 MB = 4.048 GB in 1 ms vs 5e11 flops -> HBM-bound
    r = bench.tensor_roofline(_FakeLib(5e11), _S(), 3, 512)
    assert r["bound"] == "hbm" and r["passes"] == 1
    assert r["achieved"] == pytest.approx(4.048e9 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(4.048e9 / (pk["hbm_gbs"] * 1e9) / 1e-3)
    # split TF32: three passes of 5e11 flops against the TF32 peak -> tensor-bound
    r = bench.tensor_roofline(_FakeLib(5e11), _S(), 2, 512)
    assert r["bound"] == "tensor" and r["passes"] == 3
    assert r["frac"] == pytest.approx(3 * 5e11 / (pk["tf32"] * 1e12) / 1e-3)
    assert pk["tf32"] == pytest.approx(pk["bf16"] * 1.1 / 2.25)


def test_reference_arm_line_contract():
    """`bench.py --impl reference` (the CPU oracle, as it stands) prints one JSON
    line with the contract's keys, the reference marker and zero copy bytes."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "F-applies/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""
