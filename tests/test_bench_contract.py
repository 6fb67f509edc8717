"""bench.py's reference arm (the CPU oracle) prints one JSON line with the keys
the benchmark contract asks for (CPU only; small workloads)."""
from __future__ import annotations

import json
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _run(*args):
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("args", [("--workload", "grid64"), ("--workload", "msf", "--mesh-side", "64")])
def test_reference_arm_json_line(args):
    d = _run(*args, "--steps", "2", "--warmup", "3")
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_traffic_entry_used_only_for_unchanged_sources(tmp_path, monkeypatch):
    """A committed DRAM-traffic figure fills the bench line only while the hashed kernel sources
    are unchanged; an edited source, a missing entry or a malformed file gives null."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    csrc = tmp_path / "paper_1607_05707_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("kernel a\n")
    (csrc / "b.cu").write_text("kernel b\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    entry = {"bytes_per_launch": 12345, "sources": ["a.cuh", "b.cu"], "source_sha": bench.source_sha(["a.cuh", "b.cu"])}
    tj = tmp_path / "profiles" / "traffic.json"
    tj.write_text(json.dumps({"k@w": entry}))
    assert bench.measured_traffic("k", "w") == 12345
    assert bench.measured_traffic("k", "other") is None       # keyed per workload
    assert bench.measured_traffic("other", "w") is None
    (csrc / "b.cu").write_text("kernel b, edited\n")
    assert bench.measured_traffic("k", "w") is None           # stale once a source changes
    (csrc / "b.cu").write_text("kernel b\n")
    assert bench.measured_traffic("k", "w") == 12345
    (csrc / "a.cuh").unlink()
    assert bench.measured_traffic("k", "w") is None           # a missing source
    tj.write_text("{not json")
    assert bench.measured_traffic("k", "w") is None
