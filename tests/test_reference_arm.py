"""The benchmark's reference arm (the oracle, timed on the host cores) prints
one JSON line with the contract's keys; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GTEPS" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["n_gpus"] == 1
    assert "workload" in line["config"]
    # the arms print the same config; whole steps are timed (no extrapolation): the step
    # time is the measured wall time of the timed steps
    assert line["config"]["parallelism"] == "replicas x1"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["nproc"] >= 1 and set(cb["parts_s_median"]) == {"convert", "spmv", "bfs_16_sources", "pagerank_50", "cc"}
    assert abs(line["ms_per_step"] * line["steps"] / 1e3 - cb["timed_wall_s"]) < 0.05 * cb["timed_wall_s"] + 0.05
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
