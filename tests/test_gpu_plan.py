"""Graph-captured batch plans and the batched-path autotuner against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def qstrs(p):
    return synth.packed_to_strings(np.asarray(p).reshape(-1, 3))


@pytest.mark.parametrize("path_name", ["POPC_BATCH", "TC_FP8"])
def test_plan_runs_repeatedly_with_new_queries(gpu_lib, path_name):
    fps = gpu_lib
    n = 150000
    text = synth.text(n, 81)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND)
    try:
        ks = synth.k_mix(130, seed=81)
        plan = fps.fps_batch_plan_create(lib, ks, path=getattr(fps, "FPS_PATH_" + path_name))
        try:
            for seed in (1081, 1082, 1083):
                qs = synth.packed(len(ks), seed)
                got = fps.fps_batch_plan_run(plan, qs)
                want = oracle.topk_many(text, qstrs(qs), ks)
                for (gi, gd), (wi, wd) in zip(got, want):
                    assert np.array_equal(gi, wi) and np.array_equal(gd, wd)
                # the flat form: one index / distance array laid out by the k prefix sums
                fi, fd, fc, fo = fps.fps_batch_plan_run(plan, qs, flat=True)
                assert np.array_equal(fo, fps.batch_offsets(ks))
                for q, (wi, wd) in enumerate(want):
                    assert fc[q] == len(wi)
                    assert np.array_equal(fi[fo[q]: fo[q] + fc[q]], wi) and np.array_equal(fd[fo[q]: fo[q] + fc[q]], wd)
        finally:
            fps.fps_batch_plan_release(plan)
    finally:
        fps.fps_release(lib)


def test_learned_plan_and_fallback(gpu_lib):
    fps = gpu_lib
    n = 100000
    text = synth.text(n, 82)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND)
    try:
        ks = np.full(70, 30, np.int32)
        qs = synth.packed(70, 1084)
        want = oracle.topk_many(text, qstrs(qs), ks)
        tk = np.array([w[1][-1] for w in want], np.float32)
        plan = fps.fps_batch_plan_create(lib, ks, path=fps.FPS_PATH_TC_FP8, learned=True)
        try:
            for tau, nfall in ((tk, 0), (tk - 1.0, int(np.sum(tk > 0))), (tk + 3.0, 0)):
                st = fps.fps_search_stats()
                got = fps.fps_batch_plan_run(plan, qs, tau=tau, stats=st)
                for (gi, gd), (wi, wd) in zip(got, want):
                    assert np.array_equal(gi, wi) and np.array_equal(gd, wd)
                assert st.fallbacks == nfall
                assert st.device_fallbacks == nfall          # re-run inside the graph, not by the host
        finally:
            fps.fps_batch_plan_release(plan)
    finally:
        fps.fps_release(lib)


@pytest.mark.parametrize("path_name", ["POPC_BATCH", "TC_FP8"])
def test_plan_device_fallback_on_candidate_overflow(gpu_lib, path_name):
    """60,000 copies of one record: a query equal to it accepts them all at distance 0, far more than its
    candidate region holds, so the select reports it for the exact fallback; the plan's graph re-runs it
    (WHILE node + indirect single-query scan) and the result is still the oracle's."""
    fps = gpu_lib
    x = qstrs(synth.packed(1, 1090))[0]
    rows = qstrs(synth.packed(40000, 90)) + [x] * 60000 + qstrs(synth.packed(20001, 91))
    text = synth.strings_to_text(rows)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND)
    try:
        px = fps.fps_pack_query(x)
        ks = np.array([30, 1, 1000, 10, 129, 30, 1920, 100], np.int32)
        plan = fps.fps_batch_plan_create(lib, ks, path=getattr(fps, "FPS_PATH_" + path_name))
        try:
            for rep in range(2):
                qs = synth.packed(len(ks), 1091 + rep)
                qs[[1, 4, 6]] = px                       # three overflowing queries among ordinary ones
                st = fps.fps_search_stats()
                got = fps.fps_batch_plan_run(plan, qs, stats=st)
                want = oracle.topk_many(text, qstrs(qs), ks)
                for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, want)):
                    assert np.array_equal(gi, wi) and np.array_equal(gd, wd), (rep, q)
                # k = 1 and k = 129 overflow; k = 1920's region (32 k + 8192 keys) holds the 60,000 ties
                assert st.fallbacks == st.device_fallbacks and st.device_fallbacks >= 2
        finally:
            fps.fps_batch_plan_release(plan)
    finally:
        fps.fps_release(lib)


def test_autotuner_caches_a_choice_per_size_class(gpu_lib):
    fps = gpu_lib
    n = 300000
    text = synth.text(n, 83)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND)
    try:
        for nq in (3, 200):
            seen = set()
            for seed in (1085, 1086):
                qs = synth.packed(nq, seed + nq)
                ks = synth.k_mix(nq, seed=seed)
                st = fps.fps_search_stats()
                got = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_AUTO, stats=st)
                want = oracle.topk_many(text, qstrs(qs), ks)
                for (gi, gd), (wi, wd) in zip(got, want):
                    assert np.array_equal(gi, wi) and np.array_equal(gd, wd)
                seen.add(st.path_used)
            assert seen <= {fps.FPS_PATH_POPC, fps.FPS_PATH_POPC_BATCH, fps.FPS_PATH_TC_FP8}
    finally:
        fps.fps_release(lib)
