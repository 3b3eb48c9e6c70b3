"""The benchmark's reference arm (the oracle timed on the host cores) on CPU:
rank 0 prints exactly one JSON line with the contract's keys, the line's own
figures in `cpu_baseline` and `e2e` (no host-device bytes), and the
single-thread figure beside them; any other rank prints nothing and exits 0."""
import json
import os
import subprocess
import sys

import bench


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
           "--warmup", "3", "--cpu-sample-rows", "200000"]
    return subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=bench.ROOT, env=env)


def test_reference_arm_prints_one_contract_line():
    out = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["ms_per_step"] > 0 and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and st["unit"] == "GB/s"
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    out = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
