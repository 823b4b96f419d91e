"""Pins of the batch-clustering oracle (oracle/cluster.py): its distances against the C oracle, its
silhouette against scikit-learn's and a hand-computed case, k-medoids fixed-point invariants, and planted
groups recovered with the right count."""
import numpy as np
import pytest

import oracle
import synth
from oracle import cluster


def strings(p):
    return synth.packed_to_strings(np.asarray(p).reshape(-1, 3))


def test_pair_distances_equal_the_search_oracle():
    qs = strings(synth.packed(40, 1201))
    D = cluster.pair_distances(qs)
    text = synth.strings_to_text(qs)
    for i in (0, 7, 39):
        assert D[i].tolist() == oracle.distances(text, qs[i]).tolist()
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)


def test_silhouette_matches_scikit_learn():
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(3)
    for trial in range(5):
        qs = strings(synth.packed(int(rng.integers(10, 60)), 1210 + trial))
        D = cluster.pair_distances(qs)
        for c in (2, 3, 5):
            med, lab = cluster.kmedoids(D, c)
            if len(set(lab.tolist())) < 2:
                continue
            ours = sum(cluster.silhouette_fixed(D, lab, c)) / (len(qs) * cluster.SCALE)
            ref = metrics.silhouette_score(D, lab, metric="precomputed")
            assert abs(ours - ref) <= 1e-8, (trial, c, ours, ref)


def test_silhouette_by_hand():
    # 1-D picture: A = {0, 1}, B = {10, 12} on a line, as distances
    pts = [0, 1, 10, 12]
    D = np.array([[abs(x - y) for y in pts] for x in pts])
    lab = np.array([0, 0, 1, 1])
    s = cluster.silhouette_fixed(D, lab, 2)
    # (b - a) / max(a, b): a = mean distance inside the own group, b = mean distance to the other group
    exact = [(11 - 1) / 11, (10 - 1) / 10, (9.5 - 2) / 9.5, (11.5 - 2) / 11.5]
    for got, want in zip(s, exact):
        assert abs(got / cluster.SCALE - want) < 2 ** -31
    assert s[0] == (10 * cluster.SCALE) // 11                               # floor(10/11 * 2^32)
    assert cluster.silhouette_fixed(D, np.array([0, 1, 1, 1]), 2)[0] == 0   # a singleton scores 0


def test_kmedoids_fixed_point_invariants():
    qs = strings(synth.packed(120, 1220))
    D = cluster.pair_distances(qs)
    for c in (2, 4, 7):
        med, lab = cluster.kmedoids(D, c)
        assert np.array_equal(lab, np.argmin(D[:, med], axis=1))          # everyone at its nearest medoid
        for t, m in enumerate(med):
            members = np.flatnonzero(lab == t)
            if members.size:
                cost = D[np.ix_(members, members)].sum(axis=1)
                assert D[m, members].sum() == cost.min()                    # the medoid minimises its cluster's sum


def test_planted_groups_are_recovered():
    centers = strings(synth.packed(3, 1230))
    rng = np.random.default_rng(5)
    qs, truth = [], []
    for g, ctr in enumerate(centers):
        for _ in range(15):
            b = list(ctr)
            for j in rng.choice(np.arange(1, 166), size=int(rng.integers(0, 4)), replace=False):
                b[j] = "1" if b[j] == "0" else "0"
            qs.append("".join(b))
            truth.append(g)
    res = cluster.cluster_batch(qs, 2, 8)
    assert res["c"] == 3
    lab = res["labels"]
    for g in range(3):                                                      # one label per planted group
        assert len(set(lab[np.array(truth) == g].tolist())) == 1
    assert len(set(lab.tolist())) == 3
    assert all(truth[m] == truth[np.flatnonzero(lab == lab[m])[0]] for m in res["medoids"])


def test_tiny_batches():
    qs = strings(synth.packed(2, 1240))
    assert cluster.cluster_batch(qs, 2, 8)["c"] == 1                       # no count c <= Q - 1 >= 2
    qs = strings(synth.packed(3, 1241))
    res = cluster.cluster_batch(qs, 2, 8)
    assert res["c"] == 2 and len(res["medoids"]) == 2
