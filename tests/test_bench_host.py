"""The benchmark's reference arm runs on the host (it times the CPU oracle):
its JSON line carries the keys of the benchmark contract and describes the
same workload as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-seconds", "1"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["value"] > 0 and line["unit"] == "shot-ticks/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == "toric2d_sweep" and line["config"]["points"] == 44
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert e2e["value"] == line["value"]


def test_dram_record_is_used_only_on_its_own_sources(tmp_path, monkeypatch):
    """bench.measured_traffic scales a committed DRAM record by algorithmic bytes
    and returns None once the CUDA sources differ from the ones it was taken on."""
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_2609_38139_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// kernel sources as measured\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"source_hash": bench.kernel_source_hash(), "dram_bytes": 100.0, "algorithmic_bytes": 400.0}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "batch_kernel__w__f32__dram.json").write_text(json.dumps(rec))
    assert bench.measured_traffic("w", "f32", 800.0) == 200.0
    (csrc / "k.cu").write_text("// kernel sources changed since\n")
    assert bench.measured_traffic("w", "f32", 800.0) is None
    (csrc / "k.cu").write_text("// kernel sources as measured\n")
    assert bench.measured_traffic("w", "f16", 800.0) is None
    rec["source_hash"] = "0" * 16
    (prof / "batch_kernel__w__f32__dram.json").write_text(json.dumps(rec))
    assert bench.measured_traffic("w", "f32", 800.0) is None
