"""The line bench.py prints, checked against its own contract on a short
run: the keys of the measurement contract, a roofline whose fraction is its
achieved rate over its peak with achieved = algorithmic bytes over the mean
step time, the oracle as the CPU baseline, an end-to-end figure with the
bytes it moves, a clock record and a count of the library's launches; and
the reference arm's line on the same workload and metric."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_bench_line_keeps_its_contract():
    d = _line("--steps", "5", "--warmup", "3", "--no-batched", "--no-surrogate", "--cpu-seconds", "1",
              "--e2e-inner", "2")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["dtype"] == "f32" and d["data"] == "synthetic" and "workload" in d["config"]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # value: cell-updates of the 1024^2 workload per second of the mean step
    assert d["value"] == pytest.approx(1024 * 1024 / (d["ms_per_step"] * 1e-3) / 1e6, rel=1e-6)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["algorithmic_bytes_per_launch"] == 104 * 1024 * 1024
    assert r["achieved"] == pytest.approx(r["algorithmic_bytes_per_launch"] / (d["ms_per_step"] * 1e-3) / 1e9, rel=1e-6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    assert 0.0 < r["frac"] < 1.5
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1 and c["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    # four FP64 fields in and out of pinned host memory every step
    assert e["h2d_bytes_per_step"] == 4 * 8 * 1024 * 1024 and e["d2h_bytes_per_step"] == 4 * 8 * 1024 * 1024
    assert d["gpu_launches"] >= d["steps"]
    assert d["clocks"] is None or "sm_mhz" in d["clocks"]


def test_reference_arm_times_the_oracle_on_the_same_workload():
    ours = _line("--steps", "3", "--warmup", "3", "--no-batched", "--no-surrogate", "--no-cpu-baseline",
                 "--e2e-inner", "2")
    ref = _line("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert ref["impl"] == "reference"
    for k in ("metric", "unit", "higher_is_better"):
        assert ref[k] == ours[k], k
    assert ref["config"]["workload"] == ours["config"]["workload"]
    assert ref["cpu_baseline"]["kind"] == "oracle" and ref["cpu_baseline"]["value"] == ref["value"]
    assert ref["e2e"]["h2d_bytes_per_step"] == 0 and ref["e2e"]["d2h_bytes_per_step"] == 0
