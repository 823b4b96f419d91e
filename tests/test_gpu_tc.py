"""Parity of the tensor-core batched paths (tcgen05) with the CPU oracle: 0/1 FP8 operands
(kind::f8f6f4, FP16 accumulators, 256-record tiles) and packed 0/1 FP4 operands with unit block
scales (kind::mxf4, FP32 accumulators, 128-record tiles, three accumulators).

The contraction is exact (0/1 products, integer sums <= 166, which both accumulator types
represent exactly), so the results must equal the oracle's element by element.  The ties case
(20,000 identical records) drives many accepted records through the epilogue's hand-off ring at
once.  Library sizes span one to many tiles of either format, with ragged last tiles and
buckets that end inside a tile.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

KS = [0, 1, 10, 30, 100, 129, 1000, 1920]
FORMATS = ["fp8", "fp4"]


def fmt_flags(fps, fmt):
    return fps.FPS_LOAD_TC_OPERAND if fmt == "fp8" else fps.FPS_LOAD_TC_FP4


def fmt_path(fps, fmt):
    return fps.FPS_PATH_TC_FP8 if fmt == "fp8" else fps.FPS_PATH_TC_FP4


def qstrs(packed):
    return synth.packed_to_strings(np.asarray(packed).reshape(-1, 3))


def check(fps, lib, text, qs, ks, device_io=False, fmt="fp8"):
    stats = fps.fps_search_stats()
    path = fmt_path(fps, fmt)
    if device_io:
        qd = torch.from_numpy(np.ascontiguousarray(qs).view(np.int64)).cuda()
        oi, od, oc, off = fps.fps_search_batch(lib, qd, ks, path=path)
        fps.fps_sync(lib)
        oi, od, oc = oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy()
        got = [(oi[off[q]: off[q] + oc[q]], od[off[q]: off[q] + oc[q]]) for q in range(len(ks))]
    else:
        got = fps.fps_search_batch(lib, qs, ks, path=path, stats=stats)
        assert stats.path_used == path
    want = oracle.topk_many(text, qstrs(qs), ks)
    for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, want)):
        assert len(gi) == len(wi), (q, ks[q])
        assert np.array_equal(gi, wi), (q, ks[q], gi[:8], wi[:8])
        assert np.array_equal(gd, wd), (q, ks[q])


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("n,nq", [(1, 5), (300, 130), (3000, 128), (70001, 200), (250000, 300)])
def test_tc_small_libraries(gpu_lib, n, nq, fmt):
    fps = gpu_lib
    text = synth.text(n, 41)
    lib = fps.fps_library_load(text=text, flags=fmt_flags(fps, fmt))
    try:
        info = fps.fps_library_info_get(lib)
        assert info["has_tc_operand"] == (fmt == "fp8") and info["has_tc_fp4"] == (fmt == "fp4")
        qs = np.concatenate([synth.packed(nq - 3, 1041), synth.packed_at([0, n - 1], 41),
                             np.zeros((1, 3), np.uint64)])
        ks = np.array([KS[i % len(KS)] for i in range(len(qs))], np.int32)
        check(fps, lib, text, qs, ks, fmt=fmt)
        check(fps, lib, text, qs, ks, device_io=True, fmt=fmt)
    finally:
        fps.fps_release(lib)


@pytest.mark.parametrize("fmt", FORMATS)
def test_tc_extreme_queries_and_ties(gpu_lib, fmt):
    fps = gpu_lib
    x = qstrs(synth.packed(3, 42))
    rows = [x[0]] * 20000 + qstrs(synth.packed(30000, 43)) + [x[1]] * 5000
    text = synth.strings_to_text(rows)
    lib = fps.fps_library_load(text=text, flags=fmt_flags(fps, fmt))
    try:
        qs = np.stack([np.zeros(3, np.uint64), fps.fps_pack_query("1" * 166), fps.fps_pack_query(x[0]),
                       fps.fps_pack_query(x[1])] + list(synth.packed(140, 1042)))
        ks = np.array([KS[(i + 1) % len(KS)] for i in range(len(qs))], np.int32)
        check(fps, lib, text, qs, ks, fmt=fmt)
    finally:
        fps.fps_release(lib)


def test_tc_formats_equal_popcount_batch(gpu_lib):
    fps = gpu_lib
    n = 400000
    lib = fps.fps_library_load(packed=synth.packed(n, 44), flags=fps.FPS_LOAD_TC_OPERAND | fps.FPS_LOAD_TC_FP4)
    try:
        qs = synth.packed(512, 1044)
        ks = synth.k_mix(512, seed=2)
        b = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC_BATCH)
        for path in (fps.FPS_PATH_TC_FP8, fps.FPS_PATH_TC_FP4):
            a = fps.fps_search_batch(lib, qs, ks, path=path)
            for (ai, ad), (bi, bd) in zip(a, b):
                assert np.array_equal(ai, bi) and np.array_equal(ad, bd)
    finally:
        fps.fps_release(lib)


def test_tc_operand_requires_buckets_and_int8_unsupported(gpu_lib):
    fps = gpu_lib
    with pytest.raises(fps.FpsError) as e:
        fps.fps_library_load(packed=synth.packed(100, 45), flags=fps.FPS_LOAD_TC_OPERAND | fps.FPS_LOAD_NO_BUCKETS)
    assert e.value.status == fps.FPS_ERR_UNSUPPORTED
    with pytest.raises(fps.FpsError) as e:
        fps.fps_library_load(packed=synth.packed(100, 45), flags=fps.FPS_LOAD_TC_FP4 | fps.FPS_LOAD_NO_BUCKETS)
    assert e.value.status == fps.FPS_ERR_UNSUPPORTED
    with pytest.raises(fps.FpsError) as e:
        fps.fps_library_load(packed=synth.packed(100, 45), flags=fps.FPS_LOAD_TC_INT8)
    assert e.value.status == fps.FPS_ERR_UNSUPPORTED
    lib = fps.fps_library_load(packed=synth.packed(100, 45))
    try:
        for path in (fps.FPS_PATH_TC_FP8, fps.FPS_PATH_TC_FP4):
            with pytest.raises(fps.FpsError) as e:
                fps.fps_search_batch(lib, synth.packed(2, 1045), [5, 5], path=path)
            assert e.value.status == fps.FPS_ERR_UNSUPPORTED
    finally:
        fps.fps_release(lib)


@pytest.mark.parametrize("fmt", FORMATS)
def test_tc_workload_one_million_mixed_k(gpu_lib, fmt):
    fps = gpu_lib
    n = 1_000_000
    text = synth.text_buffer(n, 0)
    lib = fps.fps_library_load(packed=synth.packed(n, 0), flags=fmt_flags(fps, fmt))
    try:
        qs = np.concatenate([synth.packed(24, synth.query_seed(2)), synth.packed_at([3, 999_999], 0)])
        ks = synth.k_mix(len(qs), seed=2)
        check(fps, lib, text, qs, ks, fmt=fmt)
    finally:
        fps.fps_release(lib)
