"""Several resident libraries searched as one (fps_search_shards) against the oracle.

The oracle sees the shards' text concatenated in global-index order (or combines per-shard oracle lists
with oracle.combine when the index bases leave gaps), so the merged result must equal the whole-library
top-k element by element.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

KS = [30, 1, 0, 1000, 10, 1920, 100, 129]


def qstrs(p):
    return synth.packed_to_strings(np.asarray(p).reshape(-1, 3))


@pytest.fixture(scope="module")
def shards(gpu_lib):
    fps = gpu_lib
    sizes, seeds = [100003, 1, 37001, 250000], [61, 62, 63, 64]
    texts = [synth.text(n, sd) for n, sd in zip(sizes, seeds)]
    libs = [fps.fps_library_load(text=t, flags=fps.FPS_LOAD_TC_OPERAND) for t in texts]
    yield fps, libs, texts, sizes
    for lb in libs:
        fps.fps_release(lb)


def queries_for(texts, sizes):
    qs = [synth.packed(50, 1061), np.zeros((1, 3), np.uint64)]
    for t, n, sd in zip(texts, sizes, [61, 62, 63, 64]):
        qs.append(synth.packed_at([0, n - 1], sd))            # records of every shard: self-matches at d = 0
    return np.concatenate(qs)


@pytest.mark.parametrize("path_name", ["POPC_BATCH", "POPC", "TC_FP8", "AUTO"])
def test_shards_equal_the_concatenated_library(shards, path_name):
    fps, libs, texts, sizes = shards
    whole = b"".join(texts)
    qs = queries_for(texts, sizes)
    ks = np.array([KS[i % len(KS)] for i in range(len(qs))], np.int32)
    want = oracle.topk_many(whole, qstrs(qs), ks)
    st = fps.fps_search_stats()
    got = fps.fps_search_shards(libs, qs, ks, path=getattr(fps, "FPS_PATH_" + path_name), stats=st)
    for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, want)):
        assert np.array_equal(gi, wi) and np.array_equal(gd, wd), (q, ks[q])
    assert st.queries == len(qs)


def test_shards_device_form_and_progress(shards):
    fps, libs, texts, sizes = shards
    whole = b"".join(texts)
    qs = queries_for(texts, sizes)
    ks = np.array([KS[(i + 3) % len(KS)] for i in range(len(qs))], np.int32)
    prog = fps.shard_progress(len(libs))
    qd = torch.from_numpy(qs.view(np.int64).copy()).cuda()
    oi, od, oc, off = fps.fps_search_shards(libs, qd, ks, path=fps.FPS_PATH_POPC_BATCH, progress=prog)
    torch.cuda.synchronize()
    for lb in libs:
        fps.fps_sync(lb)
    assert prog.tolist() == [len(qs)] * len(libs)
    oi, od, oc = oi.cpu().numpy(), od.cpu().numpy(), oc.cpu().numpy()
    want = oracle.topk_many(whole, qstrs(qs), ks)
    for q, (wi, wd) in enumerate(want):
        a = off[q]
        assert oc[q] == len(wi)
        assert np.array_equal(oi[a: a + oc[q]], wi) and np.array_equal(od[a: a + oc[q]], wd), q


def test_shards_with_index_bases_and_gaps(shards):
    fps, libs, texts, sizes = shards
    bases = [300000, 299999, 0, 500000]                       # shard 1 (one record) sits just below shard 0
    qs = queries_for(texts, sizes)[:20]
    ks = np.array([KS[i % len(KS)] for i in range(len(qs))], np.int32)
    got = fps.fps_search_shards(libs, qs, ks, index_base=bases, path=fps.FPS_PATH_POPC_BATCH)
    per = [oracle.topk_many(t, qstrs(qs), ks) for t in texts]
    for q in range(len(qs)):
        parts = [(per[s][q][0] + bases[s], per[s][q][1]) for s in range(len(libs))]
        wi, wd = oracle.combine(parts, int(ks[q]))
        gi, gd = got[q]
        assert np.array_equal(gi, wi) and np.array_equal(gd, wd), q


def test_shards_reject_overlapping_ranges_and_bad_arguments(shards):
    fps, libs, texts, sizes = shards
    qs = synth.packed(2, 1062)
    with pytest.raises(fps.FpsError) as e:
        fps.fps_search_shards(libs[:2], qs, [5, 5], index_base=[0, 100000])   # shard 1 inside shard 0's range
    assert e.value.status == fps.FPS_ERR_INVALID_ARG
    with pytest.raises(fps.FpsError) as e:
        fps.fps_search_shards(libs[:2], qs, [5, fps.FPS_K_MAX + 1])
    assert e.value.status == fps.FPS_ERR_UNSUPPORTED
