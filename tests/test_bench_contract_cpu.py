"""The benchmark's reference arm (the CPU oracle) on the host: one JSON line with the contract's keys,
the default workload's config, and silence on ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(env_extra, n=60000):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--n", str(n)], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


def test_reference_arm_line():
    lines = run_reference({"WORLD_SIZE": "1", "RANK": "0", "LOCAL_RANK": "0"})
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 1 and line["warmup"] == 1
    assert line["config"]["n_records"] == 60000 and line["config"]["k"] == 30
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_stay_silent():
    assert run_reference({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}) == []


def test_host_merge_fills_unused_slots():
    import ctypes

    import numpy as np

    import paper_1906_06170_gb300 as fps

    idx = np.array([4, 9, 1], np.int32)
    dist = np.array([2, 5, 3], np.int32)
    part = np.array([0, 2, 3], np.int64)
    oi, od = np.full(5, 7, np.int32), np.full(5, 7, np.int32)
    m = ctypes.c_int(0)
    assert fps._lib.fps_merge_topk(idx.ctypes.data, dist.ctypes.data, part.ctypes.data, 2, 5, oi.ctypes.data,
                                   od.ctypes.data, ctypes.byref(m)) == 0
    assert m.value == 3 and list(oi[:3]) == [4, 1, 9] and list(od[:3]) == [2, 3, 5]
    assert list(oi[3:]) == [-1, -1] and list(od[3:]) == [-1, -1]
