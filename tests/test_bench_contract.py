"""bench.py's reference arm (the CPU oracle timed on a bounded sample) prints one JSON line with the
keys the measurement contract asks for.  Runs on the CPU in a few seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--ref-cells", "256", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run()
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    # at least 3 warm-up steps whatever is asked (the timing rules)
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "cells/s" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_all_cores_oracle_sample():
    """The all-cores oracle sample (spawned processes, one block of cells each) reports its cores and a
    positive rate on a small mesh."""
    sys.path.insert(0, ROOT)
    import bench
    wl = dict(bench.WORKLOADS["p2-3d"], n=6)
    out = bench.cpu_baseline_all_cores(wl, bench.make_inputs(wl), 64)
    assert out["kind"] == "oracle" and out["unit"] == "cells/s"
    assert 1 <= out["cores"] <= (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
    assert out["value"] > 0 and "processes" in out["sample"]


def test_log_appends_one_record_per_run(tmp_path):
    log = tmp_path / "runs.jsonl"
    for _ in range(2):
        d = _run("--log", str(log))
    recs = [json.loads(ln) for ln in log.read_text().splitlines()]
    assert len(recs) == 2 and all(r["metric"] == d["metric"] and "logged_at" in r and "--log" in r["argv"] for r in recs)
