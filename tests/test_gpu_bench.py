"""The benchmark's GPU arm on the small 2D L = 8 workload: one JSON line with the
keys of the benchmark contract, the measured clocks and launches, the 16-bit
arms, the plain-path comparison (FP32 and int16 records identical to the plain
path's), the per-class roofline and the end-to-end rate through host buffers."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_small_workload():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "toric2d_L8_small",
                          "--steps", "2", "--warmup", "3", "--no-cpu-baseline"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e",
              "gpu_launches", "lowprec", "vs_plain", "ms_steps"):
        assert k in line, k
    assert line["value"] > 0 and line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["gpu_launches"] >= 2 and len(line["ms_steps"]) == 2
    r = line["roofline"]
    assert r["bound"] in ("hbm", "smem") and r["peak"] > 0 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert set(r["classes"]) == {"smem", "global"}
    vp = line["vs_plain"]
    assert vp["plain_f32"]["shots"] == 1000
    assert vp["batched_f32"]["identical_records"] and vp["batched_i16"]["identical_records"]
    assert set(line["lowprec"]) == {"f16", "i16"}
    e2e = line["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert line["clocks"]["sm_mhz"] is None or line["clocks"]["sm_mhz"] > 0
