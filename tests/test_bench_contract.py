"""The bench's JSON line and its traffic bookkeeping, on the CPU.

The reference arm times the FP64 oracle on the host cores, so it runs here
on a tiny sample; its line must carry every key of the bench contract.  The
traffic record of a kernel is used only while the source files that build it
are unchanged (a hash over exactly those files)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_reference_arm_line_has_the_contract_keys():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                          "--oracle-sample", "8"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "windows/s"
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["steps"] == 1 and line["n_gpus"] == 1 and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_traffic_record_follows_only_its_own_sources(tmp_path, monkeypatch):
    bench = _bench_module()
    csrc = tmp_path / "paper_1612_04787_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("// kernel a\n")
    (csrc / "b.cu").write_text("// kernel b\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    rec = {"k<256>": {"sources": ["a.cuh"], "source_hash": bench.kernel_source_hash(["a.cuh"]),
                      "dram_bytes_per_window": 1000}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("k<256>", 961) == 961000
    (csrc / "b.cu").write_text("// kernel b, changed\n")  # another kernel's file: the record stays valid
    assert bench.recorded_traffic("k<256>", 961) == 961000
    (csrc / "a.cuh").write_text("// kernel a, changed\n")  # its own source: the record no longer applies
    assert bench.recorded_traffic("k<256>", 961) is None
    assert bench.recorded_traffic("missing<256>", 961) is None
