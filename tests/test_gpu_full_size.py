"""Parity at the paper's library size: 95,417,114 generated records (Sec. 2.2), in the launch
configurations the benchmark times.

The oracle cannot scan 95 M records in seconds, so at this size every result is checked by
* the oracle, one record at a time: each returned record's distance, recomputed from its
  '0'/'1' text (Sec. 4.3), equals the returned distance;
* properties that hold at any size: min(k, N) entries per query, keys (distance, index)
  strictly ascending, indices in range;
* completeness against an independent brute force written in plain PyTorch (no kernel of
  this project): d = popc(q) + popc(x) - 2 q.x as a 0/1 FP16 matrix product, whose integer
  sums (<= 192) FP16 holds exactly, then the k smallest (d << 32 | index) keys; element by
  element, on every query of the single-query step and on a sample of the batched queries;
* agreement of the exact paths with one another (single-query scan, batched popcount,
  tensor cores, learned bounds with bad and good predictions) on every query.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from torch_brute import brute_topk

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 95_417_114
K_SINGLE, Q_SINGLE = 30, 16


@pytest.fixture(scope="module")
def full(gpu_lib):
    fps = gpu_lib
    packed = synth.packed(N, 0)
    lib = fps.fps_library_load(packed=packed, flags=fps.FPS_LOAD_TC_OPERAND | fps.FPS_LOAD_TC_FP4)
    raw = torch.from_numpy(packed.view(np.uint8).reshape(N, 24)).cuda()
    try:
        yield fps, lib, packed, raw
    finally:
        del raw
        fps.fps_release(lib)
        torch.cuda.empty_cache()


def well_formed(res, ks):
    for q, (gi, gd) in enumerate(res):
        assert len(gi) == min(int(ks[q]), N), q
        assert np.all((gi >= 0) & (gi < N)), q
        key = (gd.astype(np.int64) << 32) | gi.astype(np.int64)
        assert np.all(np.diff(key) > 0), q


def oracle_distances_agree(packed, q_row, gi, gd):
    """The oracle recomputes each returned record's distance from its text."""
    text = synth.strings_to_text(synth.packed_to_strings(packed[gi]))
    want = oracle.distances(text, synth.packed_to_strings(q_row.reshape(1, 3))[0])
    assert np.array_equal(want, gd)


def equal(res_a, res_b):
    for q, ((ai, ad), (bi, bd)) in enumerate(zip(res_a, res_b)):
        assert np.array_equal(ai, bi) and np.array_equal(ad, bd), q


def run_batch(fps, lib, qs, ks, path, tau=None):
    qd = torch.from_numpy(qs.view(np.int64).copy()).cuda()
    off = fps.batch_offsets(ks)
    oi = torch.empty(int(off[-1]), dtype=torch.int32, device="cuda")
    od = torch.empty_like(oi)
    oc = torch.empty(len(qs), dtype=torch.int32, device="cuda")
    fps.fps_search_batch(lib, qd, ks, path=path, out_index=oi, out_dist=od, out_count=oc, offsets=off,
                         tau=None if tau is None else torch.as_tensor(tau, dtype=torch.float32).cuda())
    fps.fps_sync(lib)
    oi, od, oc = oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy()
    return [(oi[off[q]: off[q] + oc[q]].copy(), od[off[q]: off[q] + oc[q]].copy()) for q in range(len(qs))]


def test_single_query_step_full_size(full):
    """The default benchmark step: 16 generated queries (seed 1001), k = 30, one after another
    through the single-query scan, device-resident inputs and outputs."""
    fps, lib, packed, raw = full
    qs = synth.packed(Q_SINGLE, 1001)
    ks = np.full(Q_SINGLE, K_SINGLE, np.int32)
    res = run_batch(fps, lib, qs, ks, fps.FPS_PATH_POPC)
    well_formed(res, ks)
    for q, (gi, gd) in enumerate(res):
        oracle_distances_agree(packed, qs[q], gi, gd)
    want = brute_topk(raw, qs, K_SINGLE)
    for q, (gi, gd) in enumerate(res):
        assert np.array_equal((gd.astype(np.int64) << 32) | gi, want[q, :K_SINGLE]), q
    # the host-buffer form (the end-to-end measurement) returns the same
    equal(fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_POPC), res)
    # extreme queries: all zeros (nearest buckets first), all ones, and a library member
    ext = np.concatenate([np.zeros((1, 3), np.uint64), synth.packed_at([N - 1], 0),
                          np.array([[~np.uint64(0), ~np.uint64(0), np.uint64((1 << 38) - 1)]], np.uint64)])
    res_e = run_batch(fps, lib, ext, np.full(3, K_SINGLE, np.int32), fps.FPS_PATH_POPC)
    want_e = brute_topk(raw, ext, K_SINGLE)
    for q, (gi, gd) in enumerate(res_e):
        assert np.array_equal((gd.astype(np.int64) << 32) | gi, want_e[q, :K_SINGLE]), q
    assert res_e[1][1][0] == 0                     # the member finds itself (or an equal record) at distance 0


def test_batched_paths_full_size(full):
    """The batched benchmark: 4096 generated queries (seed 1002), k drawn from {1, 10, 30, 100, 1000},
    on the tensor cores (FP8 and FP4 operands) and on the popcount path; a sample of 256 queries
    against the brute force."""
    fps, lib, packed, raw = full
    Q = 4096
    qs = synth.packed(Q, synth.query_seed(2))
    ks = synth.k_mix(Q, seed=2)
    tc = run_batch(fps, lib, qs, ks, fps.FPS_PATH_TC_FP8)
    well_formed(tc, ks)
    pb = run_batch(fps, lib, qs, ks, fps.FPS_PATH_POPC_BATCH)
    equal(tc, pb)
    equal(run_batch(fps, lib, qs, ks, fps.FPS_PATH_TC_FP4), pb)
    for q in range(0, Q, 8):
        oracle_distances_agree(packed, qs[q], *tc[q])
    sample = np.arange(7, Q, 16)
    want = brute_topk(raw, qs[sample], int(ks[sample].max()))
    for r, q in enumerate(sample):
        gi, gd = tc[q]
        assert np.array_equal((gd.astype(np.int64) << 32) | gi, want[r, :ks[q]]), q


def test_learned_path_full_size(full):
    """The learned-bound benchmark's search: 4096 generated queries (seed 1003), k = 30, with bounds
    that are too low, too high, random and exact; every variant equals the tensor-core path."""
    fps, lib, packed, raw = full
    Q, k = 4096, 30
    qs = synth.packed(Q, synth.query_seed(3))
    ks = np.full(Q, k, np.int32)
    ref = run_batch(fps, lib, qs, ks, fps.FPS_PATH_TC_FP8)
    well_formed(ref, ks)
    sample = np.arange(0, Q, 128)
    want = brute_topk(raw, qs[sample], k)
    for r, q in enumerate(sample):
        gi, gd = ref[q]
        assert np.array_equal((gd.astype(np.int64) << 32) | gi, want[r, :k]), q
    tk = np.array([gd[-1] for _, gd in ref], np.float32)
    rng = np.random.default_rng(11)
    for name, tau in {"exact": tk, "one_below": tk - 1.0, "random": rng.uniform(0, 40, Q).astype(np.float32),
                      "zero": np.zeros(Q, np.float32), "loose": tk + 6.0}.items():
        got = run_batch(fps, lib, qs, ks, fps.FPS_PATH_LEARNED, tau=tau)
        for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, ref)):
            assert np.array_equal(gi, wi) and np.array_equal(gd, wd), (name, q)


def test_largest_k_full_size(full):
    """k = FPS_K_MAX (1920: the single-query scan's 8-warp configuration, the largest candidate regions
    of the batched paths) at full size: every exact path equals the brute force."""
    fps, lib, packed, raw = full
    k = 1920
    qs = np.concatenate([synth.packed(2, 1005), synth.packed_at([12345], 0)])
    ks = np.full(len(qs), k, np.int32)
    want = brute_topk(raw, qs, k)
    for path in (fps.FPS_PATH_POPC, fps.FPS_PATH_POPC_BATCH, fps.FPS_PATH_TC_FP8, fps.FPS_PATH_TC_FP4):
        res = run_batch(fps, lib, qs, ks, path)
        well_formed(res, ks)
        for q, (gi, gd) in enumerate(res):
            assert np.array_equal((gd.astype(np.int64) << 32) | gi, want[q, :k]), (path, q)
    oracle_distances_agree(packed, qs[0], *res[0])
