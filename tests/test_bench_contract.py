"""bench.py prints the one-line JSON contract: the oracle arm (CPU) and the
library arm (GPU) on small grids, every required key present and consistent."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout=900):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def _common(d):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["scaling"] == "weak" and "workload" in d["config"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k


def test_reference_arm_bounded_for_many_steps():
    """A large step count shrinks the sampled window instead of the run
    growing without bound (the oracle at ~1 MLUPS on one core)."""
    import time
    t0 = time.time()
    d = _run(["--impl", "reference", "--steps", "2000", "--warmup", "3", "--ref-seconds", "10"], timeout=600)
    assert time.time() - t0 < 60
    assert d["config"]["sample_window"] < 2048 and d["steps"] == 2000


def test_reference_arm_contract():
    d = _run(["--impl", "reference", "--size", "64", "--steps", "1", "--warmup", "1", "--cpu-steps", "2"])
    _common(d)
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "64x64" in d["config"]["workload"] and d["config"]["sample_window"] <= 64


@pytest.mark.gpu
def test_library_arm_contract():
    d = _run(["--size", "256", "--steps", "20", "--warmup", "3", "--cpu-steps", "1"])
    _common(d)
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert d["gpu_launches"] == d["steps"]
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["value"] == pytest.approx(256 * 256 * d["steps"] / (d["ms_per_step"] * d["steps"] / 1e3) / 1e6, rel=1e-3)
    # both forms: the reduced state is the headline, the plain FP32 form beside it, at equal error
    f = d["forms"]
    assert d["config"]["form"] == "reduced" and set(f) >= {"reduced", "fp32", "equal_error"}
    assert f["reduced"]["MLUPS"] == d["value"] and f["reduced"]["roofline"]["bytes_per_node"] == 144
    assert f["fp32"]["roofline"]["bytes_per_node"] == 216
    assert "True" in f["equal_error"]
    assert d["speedup_vs_plain_fp32"] == pytest.approx(f["reduced"]["MLUPS"] / f["fp32"]["MLUPS"], rel=1e-3)
    assert d["cpu_baseline"]["single_core"]["cores"] == 1


def test_clock_sampler_uses_the_samples_inside_the_timed_region():
    """The clocks key is the median of the samples that arrived during the
    timed region (all samples when the region is shorter than the sampling
    interval), and counts them."""
    import time

    import bench

    c = bench.ClockSampler(0)
    c.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0,
                            "kill": lambda self: None})()
    now = time.time()
    c.lines = [(now - 0.2, "1500, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active"),
               (now + 0.05, "2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active"),
               (now + 0.5, "1600, 2070, 200.0, 0x0, Not Active, Not Active, Not Active, Not Active")]
    inside = c.stop((now, now + 0.1))
    assert inside["sm_mhz"] == 2070.0 and inside["samples_in_timed_region"] == 1
    assert inside["reasons"] == ["sw_power_cap"] and inside["samples"] == 3
    none_inside = c.stop((now + 1.0, now + 1.01))
    assert none_inside["samples_in_timed_region"] == 0 and none_inside["sm_mhz"] == 1600.0


@pytest.mark.gpu
def test_default_line_carries_the_other_workloads():
    """The default one-GPU run (the round-end form, with a short timed region)
    adds the other configurations under other_workloads, each with its own
    metric, value and roofline, and none failing."""
    d = _run(["--steps", "20", "--warmup", "3", "--no-cpu-baseline"])
    _common(d)
    o = d["other_workloads"]
    assert set(o) == {"sweep", "janus", "adjoint", "nphase", "d3q19"}
    for name, v in o.items():
        assert "error" not in v, (name, v)
        assert v["value"] > 0 and v["unit"] == "MLUPS" and "roofline" in v and "metric" in v, name
    assert set(o["janus"]["storages"]) >= {"fp32", "fp16_dev", "bf16_dev", "reduced"}
    assert set(o["sweep"]["forms"]) >= {"reduced", "fp32"}
