"""Host-side logic of bench.py: the reference arm's JSON line (the FP64
oracle on a bounded sample), its rank handling under a multi-rank launch,
and the source-hash gate on the DRAM traffic taken from a committed ncu
summary.  (The replica aggregation over gloo ranks is in
test_multirank_cpu.py.)"""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_json_line():
    r = _run(["--impl", "reference", "--workload", "2d", "--steps", "2", "--warmup", "1", "--cpu-sample", "8000"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "events/s" and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("2d")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "128x128x1" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # events per step: the sample's initialisation plus the data updates of one epoch
    assert d["config"]["events_per_step"] > 2000


def test_reference_arm_other_ranks_do_nothing():
    r = _run(["--impl", "reference", "--workload", "2d", "--steps", "1", "--warmup", "0", "--cpu-sample", "8000"],
             {"WORLD_SIZE": "2", "RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


@pytest.fixture
def bench_mod():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_profiled_traffic_follows_the_source_hash(bench_mod, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "s.txt").write_text(f"# source_sha256_16: {sha}\n# dram_bytes_per_launch: 8.85e7\n")
    monkeypatch.setattr(bench_mod, "ROOT", str(tmp_path))
    assert bench_mod.profiled_traffic("s.txt", ["k.cu"]) == 8.85e7
    src.write_bytes(b"__global__ void k() { }\n")  # the kernel changed since the capture
    assert bench_mod.profiled_traffic("s.txt", ["k.cu"]) is None
    assert bench_mod.profiled_traffic("missing.txt", ["k.cu"]) is None

