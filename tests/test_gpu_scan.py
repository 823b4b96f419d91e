"""Parity of the single-query GPU scan (FPS_PATH_POPC) with the CPU oracle.

Every comparison is element by element: same indices, same distances, same
order (ascending distance, ties by ascending index).  Integer work, so the
bar is bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def qstr(packed_row):
    return synth.packed_to_strings(np.asarray(packed_row).reshape(1, 3))[0]


def check(fps, lib, text, q_packed, k, device_io=False):
    want_i, want_d, _ = oracle.topk(text, qstr(q_packed), k)
    if device_io:
        qd = torch.from_numpy(np.asarray(q_packed, np.uint64).view(np.int64)).cuda()
        oi, od, oc = fps.fps_search_packed(lib, qd, k)
        fps.fps_sync(lib)
        c = int(oc.item())
        gi, gd = oi[:c].cpu().numpy(), od[:c].cpu().numpy()
    else:
        gi, gd = fps.fps_search_packed(lib, q_packed, k)
    assert len(gi) == len(want_i)
    assert np.array_equal(gi, want_i), (k, gi[:10], want_i[:10])
    assert np.array_equal(gd, want_d)


@pytest.mark.parametrize("n", [1, 7, 128, 129, 257, 1000, 4099, 33333])
def test_small_ragged_libraries(gpu_lib, n):
    fps = gpu_lib
    text = synth.text(n, 11)
    lib = fps.fps_library_load(text=text)
    try:
        qs = synth.packed(3, 1000 + n)
        members = synth.packed_at([0, n // 2, n - 1], 11)
        for q in list(qs) + list(members):
            for k in (1, 10, 30, 128, 129, 500):
                check(fps, lib, text, q, k)
    finally:
        fps.fps_release(lib)


@pytest.mark.parametrize("k", [1, 2, 30, 100, 128, 129, 1000, 1920])
def test_k_range_and_device_io(gpu_lib, k):
    fps = gpu_lib
    n = 60000
    text = synth.text(n, 12)
    lib = fps.fps_library_load(text=text)
    try:
        for q in synth.packed(2, 1012):
            check(fps, lib, text, q, k, device_io=False)
            check(fps, lib, text, q, k, device_io=True)
    finally:
        fps.fps_release(lib)


def test_extreme_queries_and_bucket_pruning(gpu_lib):
    fps = gpu_lib
    n = 200000
    text = synth.text(n, 13)
    lib = fps.fps_library_load(text=text)
    try:
        zeros = np.zeros(3, np.uint64)                      # Fig. 1's default query
        ones = fps.fps_pack_query("1" * 166)
        half = fps.fps_pack_query("1" * 83 + "0" * 83)
        for q in (zeros, ones, half):
            for k in (1, 30, 1000):
                check(fps, lib, text, q, k)
    finally:
        fps.fps_release(lib)


def test_no_bucket_layout(gpu_lib):
    fps = gpu_lib
    n = 50000
    text = synth.text(n, 14)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_NO_BUCKETS)
    try:
        assert not fps.fps_library_info_get(lib)["bucketed"]
        for q in list(synth.packed(2, 1014)) + [np.zeros(3, np.uint64)]:
            for k in (1, 30, 300):
                check(fps, lib, text, q, k)
    finally:
        fps.fps_release(lib)


def test_adversarial_ties(gpu_lib):
    fps = gpu_lib
    x = synth.packed_to_strings(synth.packed(3, 15))
    q = synth.packed(1, 1015)[0]
    cases = {
        "identical": [x[0]] * 70000,
        "two_alternating": [x[i % 2] for i in range(50001)],
        "three_blocks": [x[0]] * 20000 + [x[1]] * 20000 + [x[2]] * 20000,
    }
    for name, rows in cases.items():
        text = synth.strings_to_text(rows)
        lib = fps.fps_library_load(text=text)
        try:
            for k in (1, 30, 128, 1000, 1920):
                check(fps, lib, text, q, k)
            check(fps, lib, text, fps.fps_pack_query(rows[0]), 30)
        finally:
            fps.fps_release(lib)


def test_k_zero_k_above_n_and_empty_library(gpu_lib):
    fps = gpu_lib
    text = synth.text(20, 16)
    lib = fps.fps_library_load(text=text)
    try:
        q = synth.packed(1, 1016)[0]
        gi, gd = fps.fps_search_packed(lib, q, 0)
        assert len(gi) == 0
        check(fps, lib, text, q, 25)
        check(fps, lib, text, q, 1920)
        with pytest.raises(fps.FpsError):
            fps.fps_search_packed(lib, q, 1921)
        with pytest.raises(fps.FpsError):
            fps.fps_search_packed(lib, q, -1)
    finally:
        fps.fps_release(lib)
    lib = fps.fps_library_load(text=b"")
    try:
        gi, gd = fps.fps_search_packed(lib, q, 30)
        assert len(gi) == 0
    finally:
        fps.fps_release(lib)


def test_text_search_returns_cids_and_self_match(gpu_lib):
    fps = gpu_lib
    n = 5000
    rows = synth.packed_to_strings(synth.packed(n, 17))
    cids = [11050016 + 7 * i for i in range(n)]
    text = synth.strings_to_text(rows, cids=cids, sep=" ")
    lib = fps.fps_library_load(text=text)
    try:
        q = rows[1234]
        gi, gd, gc = fps.fps_search(lib, q, 30)
        wi, wd, wc = oracle.topk(text, q, 30)
        assert np.array_equal(gi, wi) and np.array_equal(gd, wd) and np.array_equal(gc, wc)
        assert gd[0] == 0 and 1234 in gi[gd == 0]           # the query itself at distance 0 (Fig. 2)
    finally:
        fps.fps_release(lib)


def test_packed_and_text_loads_agree(gpu_lib):
    fps = gpu_lib
    n = 30000
    a = synth.packed(n, 18)
    text = synth.text(n, 18)
    l1 = fps.fps_library_load(text=text)
    l2 = fps.fps_library_load(packed=a)
    try:
        for q in synth.packed(3, 1018):
            for k in (10, 200):
                i1, d1 = fps.fps_search_packed(l1, q, k)
                i2, d2 = fps.fps_search_packed(l2, q, k)
                assert np.array_equal(i1, i2) and np.array_equal(d1, d2)
        info = fps.fps_library_info_get(l2)
        assert info["n_records"] == n and info["bucket_count"].sum() == n
        bits = np.unpackbits(a.view(np.uint8), axis=1, bitorder="little")[:, :166].sum(1)
        assert np.array_equal(info["bucket_count"], np.bincount(bits, minlength=167))
    finally:
        fps.fps_release(l1)
        fps.fps_release(l2)


def test_repeated_searches_reuse_workspace(gpu_lib):
    # The scan restores its own state; 50 back-to-back searches on one stream stay exact.
    fps = gpu_lib
    n = 40000
    text = synth.text(n, 19)
    lib = fps.fps_library_load(text=text)
    try:
        qs = synth.packed(50, 1019)
        outs = []
        qd = torch.from_numpy(qs.view(np.int64)).cuda()
        for j in range(50):
            outs.append(fps.fps_search_packed(lib, qd[j], 30))
        fps.fps_sync(lib)
        want = oracle.topk_many(text, synth.packed_to_strings(qs), [30] * 50)
        for (oi, od, oc), (wi, wd) in zip(outs, want):
            assert np.array_equal(oi.cpu().numpy(), wi) and np.array_equal(od.cpu().numpy(), wd)
    finally:
        fps.fps_release(lib)


def test_workload_one_million_exact(gpu_lib):
    # 1,000,000 records of the generator (seed 0), generated queries (seed 1000), k = 30.
    fps = gpu_lib
    n = 1_000_000
    text = synth.text_buffer(n, 0)
    lib = fps.fps_library_load(packed=synth.packed(n, 0))
    try:
        for q in synth.packed(4, synth.query_seed(0)):
            check(fps, lib, text, q, 30)
        for q in synth.packed_at([5, 999_999, 123_456], 0):   # queries that are library members
            check(fps, lib, text, q, 30)
    finally:
        fps.fps_release(lib)


def test_small_library_scan_many_equal_distances(gpu_lib):
    """Libraries that take the one-wave small-library scan (up to about 1.2 M records, k <= 128)
    with so many records at one distance that a block's region cannot hold all of its records at
    its own bound: the merge then reads the records at the k-th distance again from the library
    (and, with more of them than it can sort, finds the smallest indices by bisection)."""
    fps = gpu_lib
    x = synth.packed_to_strings(synth.packed(3, 16))
    q = synth.packed(1, 1016)[0]
    cases = {
        "identical_400k": [x[0]] * 400_000,
        "identical_with_nearer_rows": [x[0]] * 150_000 + [x[1]] + [x[0]] * 150_000 + [x[2]] * 3 + [x[0]] * 50_000,
    }
    for name, rows in cases.items():
        text = synth.strings_to_text(rows)
        lib = fps.fps_library_load(text=text)
        try:
            for k in (1, 30, 128, 129):
                check(fps, lib, text, q, k)
            check(fps, lib, text, fps.fps_pack_query(rows[0]), 30, device_io=True)
        finally:
            fps.fps_release(lib)


@pytest.mark.parametrize("k", [1, 30, 128, 129])
def test_small_library_scan_at_its_size_limit(gpu_lib, k):
    """1.2 M records: the largest libraries the one-wave scan takes on 152 SMs (k <= 128), and the
    streaming scan beside it (k = 129)."""
    fps = gpu_lib
    n = 1_200_000
    text = synth.text(n, 19)
    lib = fps.fps_library_load(text=text)
    try:
        for s in (1019, 2019):
            check(fps, lib, text, synth.packed(1, s)[0], k, device_io=(s == 2019))
    finally:
        fps.fps_release(lib)
