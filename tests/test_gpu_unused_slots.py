"""Result slots past min(k, N) hold -1 on every path (the ABI's convention for k > N); slots past k
that a batched call's offsets leave free are not written.  The records before them equal the
oracle's.  Buffers start filled with a sentinel so that every write is visible."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
SENT = 7


def qstr(row):
    return synth.packed_to_strings(np.asarray(row).reshape(1, 3))[0]


def test_single_query_slots(gpu_lib):
    fps = gpu_lib
    n, k = 20, 25
    text = synth.text(n, 16)
    q = synth.packed(1, 1016)[0]
    want_i, want_d, want_c = oracle.topk(text, qstr(q), k)
    lib = fps.fps_library_load(text=text)
    try:
        # device form
        qd = torch.from_numpy(q.view(np.int64).copy()).cuda()
        oi = torch.full((k,), SENT, dtype=torch.int32, device="cuda")
        od = torch.full_like(oi, SENT)
        oc = torch.zeros(1, dtype=torch.int32, device="cuda")
        fps.fps_search_packed(lib, qd, k, out_index=oi, out_dist=od, out_count=oc)
        fps.fps_sync(lib)
        oi, od = oi.cpu().numpy(), od.cpu().numpy()
        assert int(oc.item()) == n
        assert np.array_equal(oi[:n], want_i) and np.array_equal(od[:n], want_d)
        assert np.all(oi[n:] == -1) and np.all(od[n:] == -1)
        # host form of the text call, with CIDs
        hi, hd, hc = np.full(k, SENT, np.int32), np.full(k, SENT, np.int32), np.full(k, SENT, np.int64)
        cnt = ctypes.c_int(0)
        assert fps._lib.fps_search(lib._h, qstr(q).encode(), k, hi.ctypes.data, hd.ctypes.data, hc.ctypes.data,
                                   ctypes.byref(cnt), None) == 0
        assert cnt.value == n
        assert np.array_equal(hi[:n], want_i) and np.array_equal(hd[:n], want_d) and np.array_equal(hc[:n], want_c)
        assert np.all(hi[n:] == -1) and np.all(hd[n:] == -1) and np.all(hc[n:] == -1)
        # the no-allocation entry point (same kernel, fixed scratch)
        oi2 = torch.full((k,), SENT, dtype=torch.int32, device="cuda")
        od2 = torch.full_like(oi2, SENT)
        oc2 = torch.zeros(1, dtype=torch.int32, device="cuda")
        fps.fps_search_noalloc(lib, qd, k, oi2, od2, oc2)
        fps.fps_sync(lib)
        assert int(oc2.item()) == n and torch.all(oi2[n:] == -1) and torch.all(od2[n:] == -1)
    finally:
        fps.fps_release(lib)
    # an empty library: count 0, every slot -1
    lib = fps.fps_library_load(text=b"")
    try:
        oi = torch.full((k,), SENT, dtype=torch.int32, device="cuda")
        od = torch.full_like(oi, SENT)
        oc = torch.full((1,), SENT, dtype=torch.int32, device="cuda")
        fps.fps_search_packed(lib, qd, k, out_index=oi, out_dist=od, out_count=oc)
        fps.fps_sync(lib)
        assert int(oc.item()) == 0 and torch.all(oi == -1) and torch.all(od == -1)
    finally:
        fps.fps_release(lib)


@pytest.mark.parametrize("path_name", ["POPC", "POPC_BATCH", "TC_FP8"])
def test_batch_slots_with_slack(gpu_lib, path_name):
    fps = gpu_lib
    n = 300
    text = synth.text(n, 17)
    qs = synth.packed(6, 1017)
    ks = np.array([1, 30, 299, 300, 301, 1000], np.int32)
    slack = 5                                   # free slots after every query's k
    off = np.zeros(len(ks) + 1, np.int64)
    off[1:] = np.cumsum(ks + slack)
    want = oracle.topk_many(text, synth.packed_to_strings(qs), ks)
    path = getattr(fps, "FPS_PATH_" + path_name)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND)
    try:
        # device form
        qd = torch.from_numpy(qs.view(np.int64).copy()).cuda()
        oi = torch.full((int(off[-1]),), SENT, dtype=torch.int32, device="cuda")
        od = torch.full_like(oi, SENT)
        oc = torch.zeros(len(ks), dtype=torch.int32, device="cuda")
        fps.fps_search_batch(lib, qd, ks, path=path, out_index=oi, out_dist=od, out_count=oc, offsets=off)
        fps.fps_sync(lib)
        dev = (oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy())
        # host form through the C ABI
        hi, hd = np.full(int(off[-1]), SENT, np.int32), np.full(int(off[-1]), SENT, np.int32)
        hc = np.zeros(len(ks), np.int32)
        o = fps.fps_search_opts()
        o.path = path
        assert fps._lib.fps_search_batch(lib._h, qs.ctypes.data, len(ks), ks.ctypes.data, off.ctypes.data,
                                         hi.ctypes.data, hd.ctypes.data, hc.ctypes.data, ctypes.byref(o), None) == 0
        for fi, fd, fc in (dev, (hi, hd, hc)):
            for q, (wi, wd) in enumerate(want):
                c, a = int(fc[q]), int(off[q])
                assert c == min(int(ks[q]), n)
                assert np.array_equal(fi[a: a + c], wi) and np.array_equal(fd[a: a + c], wd), (path_name, q)
                assert np.all(fi[a + c: a + ks[q]] == -1) and np.all(fd[a + c: a + ks[q]] == -1), (path_name, q)
                assert np.all(fi[a + ks[q]: off[q + 1]] == SENT) and np.all(fd[a + ks[q]: off[q + 1]] == SENT)
    finally:
        fps.fps_release(lib)


def test_shards_slots_with_slack(gpu_lib):
    fps = gpu_lib
    texts = [synth.text(120, 18), synth.text(90, 19)]
    libs = [fps.fps_library_load(text=t) for t in texts]
    try:
        qs = synth.packed(3, 1018)
        ks = np.array([30, 210, 400], np.int32)            # 210 = every record, 400 > N
        slack = 9
        off = np.zeros(len(ks) + 1, np.int64)
        off[1:] = np.cumsum(ks + slack)
        whole = texts[0] + texts[1]
        want = oracle.topk_many(whole, synth.packed_to_strings(qs), ks)
        qd = torch.from_numpy(qs.view(np.int64).copy()).cuda()
        oi = torch.full((int(off[-1]),), SENT, dtype=torch.int32, device="cuda")
        od = torch.full_like(oi, SENT)
        oc = torch.zeros(len(ks), dtype=torch.int32, device="cuda")
        fps.fps_search_shards(libs, qd, ks, out_index=oi, out_dist=od, out_count=oc, offsets=off,
                              path=fps.FPS_PATH_POPC_BATCH)
        fps.fps_sync(libs[0])
        dev = (oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy())
        hi, hd = np.full(int(off[-1]), SENT, np.int32), np.full(int(off[-1]), SENT, np.int32)
        hc = np.zeros(len(ks), np.int32)
        harr = (ctypes.c_void_p * 2)(*[lb._h for lb in libs])
        o = fps.fps_search_opts()
        o.path = fps.FPS_PATH_POPC_BATCH
        assert fps._lib.fps_search_shards(harr, 2, None, qs.ctypes.data, len(ks), ks.ctypes.data, off.ctypes.data,
                                          hi.ctypes.data, hd.ctypes.data, hc.ctypes.data, ctypes.byref(o), None,
                                          None) == 0
        for fi, fd, fc in (dev, (hi, hd, hc)):
            for q, (wi, wd) in enumerate(want):
                c, a = int(fc[q]), int(off[q])
                assert c == min(int(ks[q]), 210)                # never more than k, with free slots after k
                assert np.array_equal(fi[a: a + c], wi) and np.array_equal(fd[a: a + c], wd), q
                assert np.all(fi[a + c: a + ks[q]] == -1) and np.all(fd[a + c: a + ks[q]] == -1), q
                assert np.all(fi[a + ks[q]: off[q + 1]] == SENT) and np.all(fd[a + ks[q]: off[q + 1]] == SENT), q
    finally:
        for lb in libs:
            fps.fps_release(lb)


def test_wide_and_merge_slots(gpu_lib):
    fps = gpu_lib
    n, n_bits, k = 40, 1024, 64
    lib = fps.fps_wide_load(packed=synth.wide_packed(n, n_bits, 20), n_bits=n_bits)
    try:
        q = synth.wide_packed(1, n_bits, 1020)[0]
        for metric in (fps.FPS_METRIC_MANHATTAN, fps.FPS_METRIC_TANIMOTO):
            qd = torch.from_numpy(q.view(np.int64).copy()).cuda()
            outs = [torch.full((k,), SENT, dtype=torch.int32, device="cuda") for _ in range(3)]
            oc = torch.zeros(1, dtype=torch.int32, device="cuda")
            fps.fps_wide_search(lib, qd, k, metric, out_index=outs[0], out_num=outs[1], out_den=outs[2], out_count=oc)
            torch.cuda.synchronize()
            assert int(oc.item()) == n
            assert all(bool(torch.all(t[n:] == -1)) for t in outs)
            hs = [np.full(k, SENT, np.int32) for _ in range(3)]
            hc = np.zeros(1, np.int32)
            assert fps._lib.fps_wide_search(lib._h, q.ctypes.data, k, metric, hs[0].ctypes.data, hs[1].ctypes.data,
                                            hs[2].ctypes.data, hc.ctypes.data, 0, None) == 0
            assert int(hc[0]) == n and all(np.all(h[n:] == -1) for h in hs)
            assert np.array_equal(hs[0][:n], outs[0][:n].cpu().numpy())
    finally:
        fps.fps_wide_release(lib)
    # the host merge of shard lists: fewer records than k in all lists together
    idx = np.array([0, 5, 2], np.int32)
    dist = np.array([1, 3, 2], np.int32)
    part = np.array([0, 2, 3], np.int64)
    oi, od = np.full(6, SENT, np.int32), np.full(6, SENT, np.int32)
    m = ctypes.c_int(0)
    assert fps._lib.fps_merge_topk(idx.ctypes.data, dist.ctypes.data, part.ctypes.data, 2, 6, oi.ctypes.data,
                                   od.ctypes.data, ctypes.byref(m)) == 0
    assert m.value == 3 and list(oi[:3]) == [0, 2, 5] and list(od[:3]) == [1, 2, 3]
    assert np.all(oi[3:] == -1) and np.all(od[3:] == -1)


@pytest.mark.parametrize("path_name", ["POPC", "POPC_BATCH", "TC_FP8", "TC_FP4", "AUTO"])
def test_empty_library_batch_slots(gpu_lib, path_name):
    """A library of no records: every batched path returns count 0 and -1 in each query's k slots,
    in the device form and the host form, without launching a scan; slots past k stay untouched."""
    fps = gpu_lib
    path = getattr(fps, "FPS_PATH_" + path_name)
    lib = fps.fps_library_load(text=b"", flags=fps.FPS_LOAD_TC_OPERAND | fps.FPS_LOAD_TC_FP4)
    try:
        qs = synth.packed(4, 1023)
        ks = np.array([3, 0, 30, 7], np.int32)
        slack = 4
        off = np.zeros(len(ks) + 1, np.int64)
        off[1:] = np.cumsum(ks + slack)
        qd = torch.from_numpy(qs.view(np.int64).copy()).cuda()
        oi = torch.full((int(off[-1]),), SENT, dtype=torch.int32, device="cuda")
        od = torch.full_like(oi, SENT)
        oc = torch.full((len(ks),), SENT, dtype=torch.int32, device="cuda")
        fps.fps_search_batch(lib, qd, ks, path=path, out_index=oi, out_dist=od, out_count=oc, offsets=off)
        fps.fps_sync(lib)
        dev = (oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy())
        hi, hd = np.full(int(off[-1]), SENT, np.int32), np.full(int(off[-1]), SENT, np.int32)
        hc = np.full(len(ks), SENT, np.int32)
        o = fps.fps_search_opts()
        o.path = path
        assert fps._lib.fps_search_batch(lib._h, qs.ctypes.data, len(ks), ks.ctypes.data, off.ctypes.data,
                                         hi.ctypes.data, hd.ctypes.data, hc.ctypes.data, ctypes.byref(o), None) == 0
        for fi, fd, fc in (dev, (hi, hd, hc)):
            assert np.all(fc == 0)
            for q in range(len(ks)):
                a = int(off[q])
                assert np.all(fi[a: a + ks[q]] == -1) and np.all(fd[a: a + ks[q]] == -1), (path_name, q)
                assert np.all(fi[a + ks[q]: off[q + 1]] == SENT) and np.all(fd[a + ks[q]: off[q + 1]] == SENT)
    finally:
        fps.fps_release(lib)


def test_empty_library_plan(gpu_lib):
    """A batch plan on a library of no records: each run writes count 0 and -1 in the k slots."""
    fps = gpu_lib
    lib = fps.fps_library_load(text=b"")
    try:
        ks = np.array([5, 0, 17], np.int32)
        plan = fps.fps_batch_plan_create(lib, ks)
        try:
            qs = synth.packed(len(ks), 1024)
            for _ in range(2):
                st = fps.fps_search_stats()
                oi, od, oc, off = fps.fps_batch_plan_run(plan, qs, stats=st, flat=True)
                assert np.all(oc == 0) and st.queries == len(ks)
                assert np.all(oi[: off[-1]] == -1) and np.all(od[: off[-1]] == -1)
        finally:
            fps.fps_batch_plan_release(plan)
    finally:
        fps.fps_release(lib)
