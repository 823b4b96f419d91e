"""Host logic without a GPU: the serving loop's scheduling (fake back end), the
shard merge against the oracle's merge of the strides' lists, and the multi-rank
shard path over torch.distributed gloo (world size 2)."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def fps():
    import __graft_entry__ as ge

    ge._cuda_build_module().build()
    import paper_1906_06170_gb300 as mod

    return mod


def test_merge_topk_equals_combined_and_sorted(fps):
    rows = synth.packed_to_strings(synth.packed(6000, 61))
    q = synth.packed_to_strings(synth.packed(1, 1061))[0]
    whole = oracle.topk(synth.strings_to_text(rows), q, 50)
    for cuts in ([0, 6000], [0, 2000, 6000], [0, 1000, 1001, 3500, 6000]):
        parts = []
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            i, d, _ = oracle.topk(synth.strings_to_text(rows[lo:hi]), q, 50)
            parts.append((i + lo, d))
        mi, md = fps.fps_merge_topk(parts, 50)
        assert mi.tolist() == whole[0].tolist() and md.tolist() == whole[1].tolist()
        ci, cd = oracle.combine(parts, 50)
        assert mi.tolist() == ci.tolist()
    mi, md = fps.fps_merge_topk([(np.array([3, 9], np.int32), np.array([1, 1], np.int32))], 5)
    assert mi.tolist() == [3, 9]
    mi, md = fps.fps_merge_topk([], 5)
    assert len(mi) == 0


def test_serving_loop_schedules_every_request_once(fps):
    from paper_1906_06170_gb300 import serve

    calls = []

    def batch_fn(name, qs, ks):
        calls.append((name, len(ks)))
        return [(np.array([int(qs[i, 0] % 1000)], np.int32), np.array([int(ks[i])], np.int32)) for i in range(len(ks))]

    arr = serve.poisson_arrivals(3000, 20000.0, seed=5)
    qs = synth.packed(3000, 1062)
    names = ["1M", "20M", "95M"]
    reqs = [serve.Request(float(t), names[synth.draw(5, i, 1) % 3], qs[i], [10, 30, 100][synth.draw(5, i, 2) % 3])
            for i, t in enumerate(arr)]
    srv = serve.Server({n: None for n in names}, max_batch=64, batch_fn=batch_fn)
    done = srv.run(reqs)
    assert len(done) == 3000 and all(r.done >= r.arrival for r in done)
    assert sum(b for _, b in calls) == 3000 and max(b for _, b in calls) <= 64
    for r in done:                                   # each request got its own answer back
        assert r.result[0][0] == int(r.query[0] % 1000) and r.result[1][0] == r.k
    st = serve.latency_stats(done)
    assert st["p99_ms"] >= st["p50_ms"] >= 0 and st["throughput_rps"] > 0
    assert serve.choose_path(1, True) == fps.FPS_PATH_POPC
    assert serve.choose_path(16, True) == fps.FPS_PATH_POPC_BATCH
    assert serve.choose_path(512, False) == fps.FPS_PATH_POPC_BATCH


def test_serving_loop_multi_query_requests(fps):
    """Requests of 1..40 queries: batches hold whole requests up to max_batch queries, and every request gets
    its own results back in order."""
    from paper_1906_06170_gb300 import serve

    calls = []

    def batch_fn(name, qs, ks):
        calls.append(len(ks))
        return [(np.array([int(qs[i, 0] % 100003)], np.int32), np.array([int(ks[i])], np.int32)) for i in range(len(ks))]

    arr = serve.poisson_arrivals(300, 50000.0, seed=6)
    rng = np.random.default_rng(7)
    reqs, base = [], 0
    for i, t in enumerate(arr):
        m = int(rng.integers(1, 41))
        q = synth.packed(m, 2000 + i) if i % 3 else synth.packed(1, 2000 + i)[0]
        reqs.append(serve.Request(float(t), ["a", "b"][i % 2], q, [10, 30, 100][i % 3]))
    srv = serve.Server({"a": None, "b": None}, max_batch=64, batch_fn=batch_fn)
    done = srv.run(reqs)
    assert sum(calls) == sum(r.nq for r in done) and max(calls) <= 64
    for r in done:
        qq = np.reshape(r.query, (-1, 3))
        got = [r.result] if np.ndim(r.query) == 1 else r.result
        assert len(got) == r.nq
        for row, (gi, gd) in zip(qq, got):
            assert gi[0] == int(row[0] % 100003) and gd[0] == r.k
    st = serve.latency_stats(done)
    assert st["queries"] == sum(r.nq for r in done) and st["throughput_qps"] >= st["throughput_rps"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _shard_worker(rank, world, port, n, k, out_path):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    import paper_1906_06170_gb300 as mod

    rows = synth.packed_to_strings(synth.packed(n, 63))
    q = synth.packed_to_strings(synth.packed(1, 1063))[0]
    lo, hi = rank * n // world, (rank + 1) * n // world
    i, d, _ = orc.topk(synth.strings_to_text(rows[lo:hi]), q, k)       # this rank's shard, global indices
    mine = torch.tensor(np.stack([i + lo, d]).astype(np.int64))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.shape[1]]))
    bufs = [torch.zeros((2, int(s.item())), dtype=torch.int64) for s in sizes]
    dist.all_gather(bufs, mine)
    if rank == 0:
        parts = [(b[0].numpy().astype(np.int32), b[1].numpy().astype(np.int32)) for b in bufs]
        mi, md = mod.fps_merge_topk(parts, k)
        np.save(out_path, np.stack([mi, md]))
    dist.destroy_process_group()


def test_two_rank_shards_merge_to_global_topk(fps, tmp_path):
    import torch.multiprocessing as mp

    n, k = 5000, 40
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_shard_worker, args=(2, _free_port(), n, k, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    rows = synth.packed_to_strings(synth.packed(n, 63))
    q = synth.packed_to_strings(synth.packed(1, 1063))[0]
    wi, wd, _ = oracle.topk(synth.strings_to_text(rows), q, k)
    assert got[0].tolist() == wi.tolist() and got[1].tolist() == wd.tolist()
