"""The autotuner (FPS_PATH_AUTO) on the GPU: every (kernel, tile shape) it can choose returns the
oracle's results, its choice is written to the FPS_TUNE_CACHE file, and a fresh library of the same
size takes the cached choice without tuning."""
import json

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N = 200_000


def check(got, want):
    for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, want)):
        assert np.array_equal(gi, wi) and np.array_equal(gd, wd), q


@pytest.fixture(scope="module")
def data():
    text = synth.text(N, 61)
    qs = synth.packed(130, 1061)
    ks = synth.k_mix(130, seed=61)
    want = oracle.topk_many(text, synth.packed_to_strings(qs), ks)
    return text, qs, ks, want


def load(fps, text):
    return fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND | fps.FPS_LOAD_TC_FP4)


def test_tuning_writes_the_cache_and_a_new_library_reuses_it(gpu_lib, data, tmp_path, monkeypatch):
    fps = gpu_lib
    text, qs, ks, want = data
    cache = str(tmp_path / "tune.json")
    monkeypatch.setenv("FPS_TUNE_CACHE", cache)
    cls = fps.fps_tune_class(len(qs), int(ks.max()), False)
    lib = load(fps, text)
    try:
        st = fps.fps_search_stats()
        check(fps.fps_search_batch(lib, qs, ks, stats=st), want)     # tunes: every candidate runs
        chosen = (int(st.path_used), int(st.tile_param))
        assert chosen[0] in (fps.FPS_PATH_POPC_BATCH, fps.FPS_PATH_TC_FP8, fps.FPS_PATH_TC_FP4) and chosen[1] > 0
        entry = [e for e in json.load(open(cache))["entries"] if e["class"] == cls]
        assert len(entry) == 1 and entry[0]["n"] == N and (entry[0]["path"], entry[0]["param"]) == chosen
        st2 = fps.fps_search_stats()
        check(fps.fps_search_batch(lib, qs, ks, stats=st2), want)    # the kept choice
        assert (int(st2.path_used), int(st2.tile_param)) == chosen
    finally:
        fps.fps_release(lib)
    lib = load(fps, text)
    try:
        st3 = fps.fps_search_stats()
        check(fps.fps_search_batch(lib, qs, ks, stats=st3), want)    # read from the cache file
        assert (int(st3.path_used), int(st3.tile_param)) == chosen
    finally:
        fps.fps_release(lib)


@pytest.mark.parametrize("choice", [("POPC_BATCH", 32), ("POPC_BATCH", 128), ("TC_FP8", 32), ("TC_FP8", 128),
                                    ("TC_FP4", 48), ("TC_FP4", 192)])
def test_every_tile_shape_is_exact(gpu_lib, data, tmp_path, monkeypatch, choice):
    fps = gpu_lib
    text, qs, ks, want = data
    cache = str(tmp_path / "tune.json")
    monkeypatch.setenv("FPS_TUNE_CACHE", cache)
    lib = load(fps, text)
    try:
        path = getattr(fps, "FPS_PATH_" + choice[0])
        cls = fps.fps_tune_class(len(qs), int(ks.max()), False)
        # the device name the library keys its entries by: the one a tuned call writes
        probe = synth.packed(3, 1062)
        fps.fps_search_batch(lib, probe, [1, 2, 3])
        device = json.load(open(cache))["entries"][0]["device"]
        fps.fps_tune_cache_put(cache, device, N, cls, path, choice[1], 1.0)
    finally:
        fps.fps_release(lib)
    lib = load(fps, text)
    try:
        st = fps.fps_search_stats()
        check(fps.fps_search_batch(lib, qs, ks, stats=st), want)
        assert (int(st.path_used), int(st.tile_param)) == (path, choice[1])
    finally:
        fps.fps_release(lib)


def test_small_batches_may_choose_the_single_query_scan(gpu_lib, data, monkeypatch):
    fps = gpu_lib
    text, qs, ks, want = data
    monkeypatch.delenv("FPS_TUNE_CACHE", raising=False)
    lib = load(fps, text)
    try:
        for _ in range(2):
            st = fps.fps_search_stats()
            check(fps.fps_search_batch(lib, qs[:16], ks[:16], stats=st), want[:16])
            assert int(st.path_used) in (fps.FPS_PATH_POPC, fps.FPS_PATH_POPC_BATCH, fps.FPS_PATH_TC_FP8,
                                         fps.FPS_PATH_TC_FP4)
    finally:
        fps.fps_release(lib)
