"""The autotuner's size classes and its JSON cache file, on the host (no GPU).

A cache entry is keyed by (device name, library size N, size class) and holds the chosen batched
kernel (an fps_path code) and its tile parameter.  Round trips through the library's own reader and
writer, merges, and files written by other tools (extra keys, reordered members) are checked here;
that a cached choice returns exact results is a GPU test (test_gpu_tune.py)."""
import json

import paper_1906_06170_gb300 as fps


def test_size_classes():
    assert fps.fps_tune_class(4096, 1000, False) == "q12-k10-l0"
    assert fps.fps_tune_class(4096, 30, True) == "q12-k5-l1"
    assert fps.fps_tune_class(1, 0, False) == "q0-k0-l0"
    assert fps.fps_tune_class(16, 30, False) == "q4-k5-l0"
    assert fps.fps_tune_class(17, 31, False) == "q5-k5-l0"
    assert fps.fps_tune_class(17, 32, False) == "q5-k6-l0"


def test_cache_round_trip_and_merge(tmp_path):
    path = str(tmp_path / "tune.json")
    assert fps.fps_tune_cache_get(path, "NVIDIA GB300", 95_417_114, "q12-k10-l0") is None
    fps.fps_tune_cache_put(path, "NVIDIA GB300", 95_417_114, "q12-k10-l0", fps.FPS_PATH_TC_FP4, 96, 30.25)
    fps.fps_tune_cache_put(path, "NVIDIA GB300", 95_417_114, "q4-k5-l0", fps.FPS_PATH_POPC, 0, 5.5)
    fps.fps_tune_cache_put(path, "NVIDIA GB300", 1_000_000, "q12-k10-l0", fps.FPS_PATH_POPC_BATCH, 128, 1.5)
    fps.fps_tune_cache_put(path, 'dev "quoted" \\ name', 7, "q0-k0-l0", fps.FPS_PATH_TC_FP8, 32, 0.125)
    assert fps.fps_tune_cache_get(path, "NVIDIA GB300", 95_417_114, "q12-k10-l0") == (fps.FPS_PATH_TC_FP4, 96, 30.25)
    assert fps.fps_tune_cache_get(path, "NVIDIA GB300", 95_417_114, "q4-k5-l0") == (fps.FPS_PATH_POPC, 0, 5.5)
    assert fps.fps_tune_cache_get(path, "NVIDIA GB300", 1_000_000, "q12-k10-l0") == (fps.FPS_PATH_POPC_BATCH, 128, 1.5)
    assert fps.fps_tune_cache_get(path, 'dev "quoted" \\ name', 7, "q0-k0-l0") == (fps.FPS_PATH_TC_FP8, 32, 0.125)
    assert fps.fps_tune_cache_get(path, "NVIDIA GB300", 95_417_114, "q12-k10-l1") is None
    assert fps.fps_tune_cache_get(path, "other", 95_417_114, "q12-k10-l0") is None
    # a new choice for a known key replaces the old one; the other entries stay
    fps.fps_tune_cache_put(path, "NVIDIA GB300", 95_417_114, "q12-k10-l0", fps.FPS_PATH_TC_FP8, 128, 29.0)
    assert fps.fps_tune_cache_get(path, "NVIDIA GB300", 95_417_114, "q12-k10-l0") == (fps.FPS_PATH_TC_FP8, 128, 29.0)
    doc = json.load(open(path))          # the file is plain JSON
    assert doc["fps_tune_cache"] == 1 and len(doc["entries"]) == 4
    assert doc["entries"][3]["device"] == 'dev "quoted" \\ name'


def test_cache_written_by_another_tool(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"note": {"a": [1, 2, {"b": None}]}, "fps_tune_cache": 1, "entries": [
        {"ms": 2.0, "param": 64, "path": 2, "class": "q10-k7-l0", "n": 1000, "device": "X", "extra": [True]},
        {"device": "X", "n": 1000, "class": "incomplete"}]}, indent=2))
    assert fps.fps_tune_cache_get(str(path), "X", 1000, "q10-k7-l0") == (fps.FPS_PATH_POPC_BATCH, 64, 2.0)
    assert fps.fps_tune_cache_get(str(path), "X", 1000, "incomplete") is None


def test_unreadable_cache_is_replaced(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert fps.fps_tune_cache_get(str(path), "X", 1, "q0-k0-l0") is None
    fps.fps_tune_cache_put(str(path), "X", 1, "q0-k0-l0", fps.FPS_PATH_POPC, 0, 1.0)
    assert fps.fps_tune_cache_get(str(path), "X", 1, "q0-k0-l0") == (fps.FPS_PATH_POPC, 0, 1.0)
