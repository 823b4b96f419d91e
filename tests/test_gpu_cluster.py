"""Batch clustering search on the GPU (fps_cluster_search) against oracle/cluster.py and the search oracle:
the chosen count, the silhouette scores of every count, the labels, the medoids and each cluster's top-k
must all be identical."""
import numpy as np
import pytest

import oracle
import synth
from oracle import cluster

pytestmark = pytest.mark.gpu


def strings(p):
    return synth.packed_to_strings(np.asarray(p).reshape(-1, 3))


def planted_batch(n_groups, per_group, seed, flips=4):
    centers = synth.packed(n_groups, seed)
    rng = np.random.default_rng(seed)
    out = []
    for g in range(n_groups):
        for _ in range(per_group):
            x = centers[g].copy()
            for j in rng.choice(np.arange(1, 166), size=int(rng.integers(0, flips + 1)), replace=False):
                x[j // 64] ^= np.uint64(1) << np.uint64(j % 64)
            out.append(x)
    return np.stack(out)


def check(fps, lib, text, qs, k, c_min, c_max):
    got = fps.fps_cluster_search(lib, qs, k=k, c_min=c_min, c_max=c_max)
    want = cluster.cluster_batch(strings(qs), c_min, c_max)
    assert got["c"] == want["c"]
    assert got["scores"] == want["scores"]
    assert got["medoids"].tolist() == list(want["medoids"])
    assert got["labels"].tolist() == [int(x) for x in want["labels"]]
    for t, m in enumerate(want["medoids"]):
        wi, wd, _ = oracle.topk(text, strings(qs[m])[0], k)
        gi, gd = got["results"][t]
        assert gi.tolist() == wi.tolist() and gd.tolist() == wd.tolist()
    return got


@pytest.fixture(scope="module")
def library(gpu_lib):
    fps = gpu_lib
    text = synth.text(150000, 120)
    lib = fps.fps_library_load(text=text)
    yield fps, lib, text
    fps.fps_release(lib)


@pytest.mark.parametrize("Q", [1, 2, 3, 17, 64, 300])
def test_cluster_search_random_batches(library, Q):
    fps, lib, text = library
    check(fps, lib, text, synth.packed(Q, 1300 + Q), 30, 2, 8)


def test_cluster_search_planted_groups(library):
    fps, lib, text = library
    qs = planted_batch(5, 40, 1350)
    got = check(fps, lib, text, qs, 30, 2, 10)
    assert got["c"] == 5
    for g in range(5):
        assert len(set(got["labels"][40 * g: 40 * (g + 1)].tolist())) == 1


def test_cluster_search_duplicates_large_batch_and_k(library):
    fps, lib, text = library
    qs = np.concatenate([planted_batch(3, 300, 1360, flips=2), np.repeat(synth.packed(1, 1361), 200, axis=0),
                         synth.packed(500, 1362)])
    check(fps, lib, text, qs, 1000, 2, 16)
    check(fps, lib, text, qs[:50], 0, 3, 5)


def test_cluster_search_argument_errors(library):
    fps, lib, text = library
    qs = synth.packed(10, 1370)
    for kw in ({"c_min": 1}, {"c_min": 5, "c_max": 4}, {"c_max": 17}):
        with pytest.raises(fps.FpsError) as e:
            fps.fps_cluster_search(lib, qs, **kw)
        assert e.value.status == fps.FPS_ERR_INVALID_ARG
    with pytest.raises(fps.FpsError) as e:
        fps.fps_cluster_search(lib, synth.packed(fps.FPS_CLUSTER_MAX_Q + 1, 1371))
    assert e.value.status == fps.FPS_ERR_INVALID_ARG
