"""Concurrent searches on one library: every CUDA stream gets its own workspace (scan states, staging), so
work interleaved on two streams, and two host threads each with its own stream, must all return the
oracle's results."""
import threading

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def qstrs(p):
    return synth.packed_to_strings(np.asarray(p).reshape(-1, 3))


@pytest.fixture(scope="module")
def lib_text(gpu_lib):
    fps = gpu_lib
    text = synth.text(250000, 140)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND)
    yield fps, lib, text
    fps.fps_release(lib)


def unpack(oi, od, oc, off, Q):
    oi, od, oc = oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy()
    return [(oi[off[q]: off[q] + oc[q]], od[off[q]: off[q] + oc[q]]) for q in range(Q)]


def test_two_streams_interleaved(lib_text):
    fps, lib, text = lib_text
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    qa, qb = synth.packed(40, 1401), synth.packed(150, 1402)
    ka, kb = synth.k_mix(40, seed=4), synth.k_mix(150, seed=5)
    wa = oracle.topk_many(text, qstrs(qa), ka)
    wb = oracle.topk_many(text, qstrs(qb), kb)
    qs1 = synth.packed(6, 1403)
    w1 = [oracle.topk(text, s, 30)[:2] for s in qstrs(qs1)]
    da = torch.from_numpy(qa.view(np.int64).copy()).cuda()
    db = torch.from_numpy(qb.view(np.int64).copy()).cuda()
    d1 = torch.from_numpy(qs1.view(np.int64).copy()).cuda()
    torch.cuda.synchronize()
    for rep in range(3):
        ra = fps.fps_search_batch(lib, da, ka, path=fps.FPS_PATH_POPC, stream=s1)        # chained single scans
        singles = [fps.fps_search_packed(lib, d1[j], 30, stream=s2) for j in range(len(qs1))]
        rb = fps.fps_search_batch(lib, db, kb, path=fps.FPS_PATH_TC_FP8, stream=s2)
        rc = fps.fps_search_batch(lib, db[:40], kb[:40], path=fps.FPS_PATH_POPC_BATCH, stream=s1)
        s1.synchronize()
        s2.synchronize()
        fps.fps_sync(lib, s1)
        fps.fps_sync(lib, s2)
        for (gi, gd), (wi, wd) in zip(unpack(*ra[:3], ra[3], len(ka)), wa):
            assert np.array_equal(gi, wi) and np.array_equal(gd, wd), rep
        for (gi, gd), (wi, wd) in zip(unpack(*rb[:3], rb[3], len(kb)), wb):
            assert np.array_equal(gi, wi) and np.array_equal(gd, wd), rep
        for (gi, gd), (wi, wd) in zip(unpack(*rc[:3], rc[3], 40), wb[:40]):
            assert np.array_equal(gi, wi) and np.array_equal(gd, wd), rep
        for (oi, od, oc), (wi, wd) in zip(singles, w1):
            c = int(oc.item())
            assert oi[:c].cpu().tolist() == wi.tolist() and od[:c].cpu().tolist() == wd.tolist(), rep


def test_two_host_threads_each_with_a_stream(lib_text):
    fps, lib, text = lib_text
    qs = [synth.packed(60, 1410 + t) for t in range(2)]
    ks = [synth.k_mix(60, seed=10 + t) for t in range(2)]
    want = [oracle.topk_many(text, qstrs(q), k) for q, k in zip(qs, ks)]
    errors = []

    def work(t):
        try:
            st = torch.cuda.Stream()
            for rep in range(4):
                path = fps.FPS_PATH_POPC_BATCH if (rep + t) % 2 else fps.FPS_PATH_POPC
                got = fps.fps_search_batch(lib, qs[t], ks[t], path=path, stream=st)
                for (gi, gd), (wi, wd) in zip(got, want[t]):
                    if not (np.array_equal(gi, wi) and np.array_equal(gd, wd)):
                        errors.append((t, rep))
                        return
        except Exception as e:   # reported by the main thread
            errors.append((t, repr(e)))

    th = [threading.Thread(target=work, args=(t,)) for t in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
