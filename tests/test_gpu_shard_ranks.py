"""The library split across ranks (the paper's strides searched apart, their lists merged and sorted
again; Sec. 2.1 and the text after Fig. 3), with the product's own search on every rank.

Two processes each load one contiguous half of the library on the GPU and search it with the batched
entry point (mixed k); the per-query lists, with global indices, travel to rank 0 through a gloo
all-gather, where fps_merge_topk merges them.  The merged lists must equal the oracle's top-k over the
whole library.  The two ranks' kernels never wait on each other: each rank's searches finish on its
own before the exchange, which runs on the host."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N, Q = 60_000, 12
KS = np.array([1, 10, 30, 100, 1000, 5, 30, 30, 64, 2, 300, 30], np.int32)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, path_code, out_path):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1906_06170_gb300 as fps

    torch.cuda.set_device(0)
    lo, hi = rank * N // world, (rank + 1) * N // world
    lib = fps.fps_library_load(packed=synth.packed(hi - lo, 64, start=lo),
                               flags=fps.FPS_LOAD_TC_OPERAND | fps.FPS_LOAD_TC_FP4)
    try:
        res = fps.fps_search_batch(lib, synth.packed(Q, 1064), KS, path=path_code)
    finally:
        fps.fps_release(lib)
    # this rank's lists with global indices: [query, index, distance] rows
    mine = torch.tensor(np.concatenate([np.stack([np.full(len(i), q), i + lo, d]) for q, (i, d) in enumerate(res)],
                                       axis=1).astype(np.int64))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.shape[1]]))
    bufs = [torch.zeros((3, int(s.item())), dtype=torch.int64) for s in sizes]
    dist.all_gather(bufs, mine)
    if rank == 0:
        merged = {}
        for q in range(Q):
            parts = [(b[1][b[0] == q].numpy().astype(np.int32), b[2][b[0] == q].numpy().astype(np.int32))
                     for b in bufs]
            merged[f"i{q}"], merged[f"d{q}"] = fps.fps_merge_topk(parts, int(KS[q]))
        np.savez(out_path, **merged)
    dist.destroy_process_group()


@pytest.mark.parametrize("path_name", ["POPC", "AUTO", "TC_FP4"])
def test_two_ranks_search_their_halves_and_merge(gpu_lib, tmp_path, path_name):
    import torch.multiprocessing as mp

    fps = gpu_lib
    out = str(tmp_path / "merged.npz")
    mp.start_processes(_rank, args=(2, _free_port(), getattr(fps, "FPS_PATH_" + path_name), out), nprocs=2,
                       join=True, start_method="spawn")
    got = np.load(out)
    text = synth.text(N, 64)
    want = oracle.topk_many(text, synth.packed_to_strings(synth.packed(Q, 1064)), KS)
    for q in range(Q):
        assert got[f"i{q}"].tolist() == want[q][0].tolist(), q
        assert got[f"d{q}"].tolist() == want[q][1].tolist(), q
