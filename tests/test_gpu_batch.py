"""Parity of the batched search paths with the CPU oracle (element by element)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

KS = [0, 1, 10, 30, 100, 129, 1000, 1920]


def qstrs(packed):
    return synth.packed_to_strings(np.asarray(packed).reshape(-1, 3))


def run_batch(fps, lib, queries, ks, path, device_io):
    if device_io:
        qd = torch.from_numpy(np.ascontiguousarray(queries).view(np.int64)).cuda()
        oi, od, oc, off = fps.fps_search_batch(lib, qd, ks, path=path)
        fps.fps_sync(lib)
        oi, od, oc = oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy()
        return [(oi[off[q]: off[q] + oc[q]], od[off[q]: off[q] + oc[q]]) for q in range(len(ks))]
    return fps.fps_search_batch(lib, queries, ks, path=path)


def check_batch(fps, lib, text, queries, ks, path, device_io=False):
    got = run_batch(fps, lib, queries, ks, path, device_io)
    want = oracle.topk_many(text, qstrs(queries), ks)
    for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, want)):
        assert len(gi) == len(wi), (q, ks[q])
        assert np.array_equal(gi, wi), (q, ks[q], gi[:8], wi[:8])
        assert np.array_equal(gd, wd), (q, ks[q])


@pytest.mark.parametrize("n", [1, 7, 1000, 33333, 200000])
def test_batch_popc_small_libraries(gpu_lib, n):
    fps = gpu_lib
    text = synth.text(n, 31)
    lib = fps.fps_library_load(text=text)
    try:
        qs = np.concatenate([synth.packed(16, 1031), synth.packed_at([0, n // 3, n - 1], 31),
                             np.zeros((1, 3), np.uint64)])
        ks = np.array([KS[i % len(KS)] for i in range(len(qs))], np.int32)
        check_batch(fps, lib, text, qs, ks, fps.FPS_PATH_POPC_BATCH)
        check_batch(fps, lib, text, qs, ks, fps.FPS_PATH_POPC_BATCH, device_io=True)
        check_batch(fps, lib, text, qs, ks, fps.FPS_PATH_AUTO)
        # the flat host form returns the same records without per-query copies (k may exceed n)
        lists = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC_BATCH)
        fi, fd, fc, fo = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC_BATCH, flat=True)
        for q, (gi, gd) in enumerate(lists):
            assert fc[q] == len(gi) == min(int(ks[q]), n)
            assert np.array_equal(fi[fo[q]: fo[q] + fc[q]], gi) and np.array_equal(fd[fo[q]: fo[q] + fc[q]], gd)
    finally:
        fps.fps_release(lib)


def test_batch_overflow_falls_back_exactly(gpu_lib):
    fps = gpu_lib
    x = qstrs(synth.packed(2, 32))
    rows = [x[0]] * 60000 + [x[1]] * 3000        # massive ties: candidate regions overflow
    text = synth.strings_to_text(rows)
    lib = fps.fps_library_load(text=text)
    try:
        qs = np.concatenate([synth.packed(3, 1032), fps.fps_pack_query(x[1]).reshape(1, 3)])
        ks = np.array([30, 1, 1000, 100], np.int32)
        stats = fps.fps_search_stats()
        got = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC_BATCH, stats=stats)
        want = oracle.topk_many(text, qstrs(qs), ks)
        for (gi, gd), (wi, wd) in zip(got, want):
            assert np.array_equal(gi, wi) and np.array_equal(gd, wd)
        assert stats.fallbacks >= 1
        check_batch(fps, lib, text, qs, ks, fps.FPS_PATH_POPC_BATCH, device_io=True)
    finally:
        fps.fps_release(lib)


def test_batch_equals_sequential_single_queries(gpu_lib):
    fps = gpu_lib
    n = 120000
    lib = fps.fps_library_load(packed=synth.packed(n, 33))
    try:
        qs = synth.packed(40, 1033)
        ks = synth.k_mix(40, seed=2)
        a = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC_BATCH)
        b = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC)
        for (ai, ad), (bi, bd) in zip(a, b):
            assert np.array_equal(ai, bi) and np.array_equal(ad, bd)
    finally:
        fps.fps_release(lib)


def test_batch_workload_one_million_mixed_k(gpu_lib):
    # 1,000,000 generated records (seed 0), 24 queries, k from {1, 10, 30, 100, 1000}
    fps = gpu_lib
    n = 1_000_000
    text = synth.text_buffer(n, 0)
    lib = fps.fps_library_load(packed=synth.packed(n, 0))
    try:
        qs = np.concatenate([synth.packed(20, synth.query_seed(2)), synth.packed_at([1, 500_000, 999_998, 77], 0)])
        ks = synth.k_mix(len(qs), seed=2)
        check_batch(fps, lib, text, qs, ks, fps.FPS_PATH_POPC_BATCH)
    finally:
        fps.fps_release(lib)


def test_sequential_chain_alternates_states_exactly(gpu_lib):
    """FPS_PATH_POPC runs the queries one after another, each launch after the first a programmatic
    dependent of the previous one on the other scan state.  Mixed k switches between the two kernel
    configurations inside the chain, k = 0 entries are skipped, a run of equal records forces the
    merge's bisection path mid-chain, and repeated calls plus a single search afterwards reuse both
    states."""
    fps = gpu_lib
    x = qstrs(synth.packed(2, 1040))
    rows = qstrs(synth.packed(150000, 40)) + [x[0]] * 20000 + qstrs(synth.packed(30001, 41))
    text = synth.strings_to_text(rows)
    lib = fps.fps_library_load(text=text)
    try:
        qs = np.concatenate([synth.packed(21, 1041), np.stack([fps.fps_pack_query(x[0])] * 3)])
        cyc = [30, 0, 1, 1920, 100, 129, 10, 1000]
        ks = np.array([cyc[i % len(cyc)] for i in range(len(qs))], np.int32)
        want = oracle.topk_many(text, qstrs(qs), ks)
        for rep in range(2):
            got = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC)
            for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, want)):
                assert np.array_equal(gi, wi) and np.array_equal(gd, wd), (rep, q, ks[q])
        check_batch(fps, lib, text, qs, ks, fps.FPS_PATH_POPC, device_io=True)
        gi, gd = fps.fps_search_packed(lib, qs[3], 50)
        wi, wd, _ = oracle.topk(text, qstrs(qs[3:4])[0], 50)
        assert np.array_equal(gi, wi) and np.array_equal(gd, wd)
    finally:
        fps.fps_release(lib)
