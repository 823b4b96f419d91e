"""Serving loop on the GPU: dynamic batches give exactly the per-request answers;
libraries are admitted by device-memory budget."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_batched_serving_matches_per_request_search(gpu_lib):
    fps = gpu_lib
    from paper_1906_06170_gb300 import serve

    sizes = {"small": (50_000, 10), "mid": (200_000, 11), "large": (600_000, 12)}
    libs = {nm: fps.fps_library_load(packed=synth.packed(n, s), flags=fps.FPS_LOAD_TC_OPERAND)
            for nm, (n, s) in sizes.items()}
    try:
        arr = serve.poisson_arrivals(1500, 5000.0, seed=5)
        qs = synth.packed(1500, 1071)
        names = list(sizes)
        reqs = [serve.Request(float(t), names[synth.draw(5, i, 1) % 3], qs[i], [10, 30, 100][synth.draw(5, i, 2) % 3])
                for i, t in enumerate(arr)]
        srv = serve.Server(libs, has_tc={nm: True for nm in names}, max_batch=512)
        done = srv.run(reqs)
        for r in done:
            wi, wd = fps.fps_search_packed(libs[r.lib], r.query, r.k)
            assert np.array_equal(r.result[0], wi) and np.array_equal(r.result[1], wd)
        st = serve.latency_stats(done)
        assert st["requests"] == 1500 and st["p99_ms"] >= st["p50_ms"]
    finally:
        for lib in libs.values():
            fps.fps_release(lib)


def test_libraries_admitted_by_device_budget(gpu_lib):
    fps = gpu_lib
    packed = synth.packed(300_000, 13)
    lib = fps.fps_library_load(packed=packed)
    need = fps.fps_library_info_get(lib)["device_bytes"]
    fps.fps_release(lib)
    with pytest.raises(fps.FpsError) as e:
        fps.fps_library_load(packed=packed, hbm_budget_bytes=need - 1)
    assert e.value.status == fps.FPS_ERR_BUDGET
    lib = fps.fps_library_load(packed=packed, hbm_budget_bytes=need)
    fps.fps_release(lib)
