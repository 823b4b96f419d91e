"""The allocation-free single-query search, through the C ABI, against the regular search and the oracle.

fps_search_noalloc serves callers that cannot allocate device memory while
searching: code whose device memory is all owned by another allocator, code
whose latency budget cannot take a cudaMalloc and its synchronisation, code that
searches on many short-lived streams (each would get its own workspace).  It
keeps its scratch in a fixed array inside the library, shared by every call on a
device, so consecutive calls must each start clean: its results must equal
fps_search_packed's and the oracle's exactly (integer outputs) call after call,
also right after a call that failed on the device.  This file is named to be
collected last.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
SENT = -7


def _noalloc(fps, lib, qd, k):
    oi = torch.full((max(k, 1),), SENT, dtype=torch.int32, device="cuda")
    od = torch.full_like(oi, SENT)
    oc = torch.full((1,), SENT, dtype=torch.int32, device="cuda")
    fps.fps_search_noalloc(lib, qd, k, oi, od, oc)
    torch.cuda.synchronize()
    fps.fps_sync(lib)
    return oi.cpu().numpy(), od.cpu().numpy(), int(oc.item())


def test_noalloc_matches_regular_search_and_oracle_on_consecutive_calls(gpu_lib):
    fps = gpu_lib
    n = 300_000
    text = synth.text(n, 21)
    qs = synth.packed(4, 1021)
    qstrs = synth.packed_to_strings(qs)
    lib = fps.fps_library_load(text=text)
    try:
        qd = torch.from_numpy(qs.view(np.int64).copy()).cuda()
        for k in (30, 1, 128):
            for j in (0, 1, 1, 2):                   # two different queries in a row, then a repeat
                want_i, want_d, _ = oracle.topk(text, qstrs[j], k)
                reg_i, reg_d, reg_c = fps.fps_search_packed(lib, qd[j], k)
                oi, od, c = _noalloc(fps, lib, qd[j], k)
                assert c == int(reg_c.item()) == min(k, n)
                assert np.array_equal(oi[:c], want_i) and np.array_equal(od[:c], want_d)
                assert np.array_equal(oi[:c], reg_i.cpu().numpy()[:c])
                assert np.array_equal(od[:c], reg_d.cpu().numpy()[:c])
        oi = torch.empty(256, dtype=torch.int32, device="cuda")
        with pytest.raises(fps.FpsError) as e:
            fps.fps_search_noalloc(lib, qd[0], fps.FPS_NOALLOC_K_MAX + 1, oi, oi, oi)
        assert e.value.status == fps.FPS_ERR_UNSUPPORTED
    finally:
        fps.fps_release(lib)


def test_noalloc_k_above_n_and_empty_library(gpu_lib):
    fps = gpu_lib
    n, k = 20, 30
    text = synth.text(n, 22)
    q = synth.packed(1, 1022)
    want_i, want_d, _ = oracle.topk(text, synth.packed_to_strings(q)[0], k)
    qd = torch.from_numpy(q[0].view(np.int64).copy()).cuda()
    lib = fps.fps_library_load(text=text)
    try:
        for _ in range(2):
            oi, od, c = _noalloc(fps, lib, qd, k)
            assert c == n
            assert np.array_equal(oi[:n], want_i) and np.array_equal(od[:n], want_d)
            assert np.all(oi[n:k] == -1) and np.all(od[n:k] == -1)
    finally:
        fps.fps_release(lib)
    lib = fps.fps_library_load(text=b"")
    try:
        oi, od, c = _noalloc(fps, lib, qd, k)
        assert c == 0 and np.all(oi[:k] == -1) and np.all(od[:k] == -1)
        oi, od, c = _noalloc(fps, lib, qd, 0)
        assert c == 0
    finally:
        fps.fps_release(lib)


def test_noalloc_device_failure_reported_then_next_call_exact(gpu_lib, monkeypatch):
    # A 20 M-record library streams ~70 tiles per warp, so with a 1 ns bound on each wait some
    # wait is still pending after the deadline: the call reports *out_count = -1.  The scratch it
    # leaves behind must not change the next call's results.
    fps = gpu_lib
    n, k = 20_000_000, 30
    lib = fps.fps_library_load(packed=synth.packed(n, 30))
    try:
        q = synth.packed(2, 1030)
        qd = torch.from_numpy(q.view(np.int64).copy()).cuda()
        monkeypatch.setenv("FPS_NOALLOC_TIMEOUT_NS", "1")
        _, _, c = _noalloc(fps, lib, qd[0], k)
        assert c == -1
        monkeypatch.delenv("FPS_NOALLOC_TIMEOUT_NS")
        for j in (0, 1):
            reg_i, reg_d, reg_c = fps.fps_search_packed(lib, qd[j], k)
            oi, od, c = _noalloc(fps, lib, qd[j], k)
            assert c == int(reg_c.item()) == k
            assert np.array_equal(oi[:k], reg_i.cpu().numpy()) and np.array_equal(od[:k], reg_d.cpu().numpy())
    finally:
        os.environ.pop("FPS_NOALLOC_TIMEOUT_NS", None)
        fps.fps_release(lib)
