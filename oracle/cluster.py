"""Oracle of the batch clustering search -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU legs may use this
module; the CUDA path never imports it.

The paper's interface offers a "batch clustering search" (Sec. 4.4 and the
results shown after Fig. 1): a batch of query fingerprints is clustered, the
number of clusters is chosen by the silhouette ("contour") coefficient, and the
top 30 library molecules are listed per cluster.  The paper names neither the
clustering algorithm nor what a cluster is searched with; the readings here
(one deterministic procedure, exact integer arithmetic) are:

* distance between two queries: the Manhattan distance of Sec. 4.3;
* clustering for a given count c: k-medoids.  First medoid: the query with the
  smallest sum of distances to all queries; each further medoid: the query
  farthest from its nearest chosen medoid (farthest-first).  Then alternate
  (at most MAX_ITER rounds, stopping when the medoids repeat): assign every
  query to its nearest medoid (ties: the medoid chosen first), and make the
  member with the smallest sum of distances to its cluster the new medoid.
  Ties between queries always go to the smaller query index;
* silhouette of query i in cluster A: a = mean distance to the other members
  of A, b = the smallest mean distance to the members of another non-empty
  cluster, s = (b - a) / max(a, b) (0 when max(a, b) = 0 or |A| = 1).  Kept
  exactly as the integer floor(s * 2^32); a clustering's score is the sum over
  queries (the mean times Q * 2^32);
* the count is the c in [c_min, c_max] with the largest score (ties: smaller c);
* every cluster of the chosen clustering is searched with its medoid: the k
  nearest library records by (distance, index), as in the single-molecule search.
"""
from __future__ import annotations

import numpy as np

MAX_ITER = 30
SCALE = 1 << 32


def pair_distances(q_strings):
    """D[i][j] = Manhattan distance of queries i and j (character compares, Sec. 4.3)."""
    a = np.array([[c == "1" for c in s] for s in q_strings], dtype=np.int64)
    return (a[:, None, :] != a[None, :, :]).sum(axis=2)


def first_medoids(D, c):
    Q = D.shape[0]
    med = [int(np.argmin(D.sum(axis=1)))]          # argmin returns the smallest index among ties
    near = D[:, med[0]].copy()
    for _ in range(1, c):
        far = near.copy()
        far[med] = -1                              # a chosen medoid is never chosen again
        m = int(np.argmax(far))
        med.append(m)
        near = np.minimum(near, D[:, m])
    return med


def assign(D, med):
    """Nearest medoid of every query; ties go to the medoid chosen first."""
    return np.argmin(D[:, med], axis=1)


def kmedoids(D, c):
    med = first_medoids(D, c)
    for _ in range(MAX_ITER):
        lab = assign(D, med)
        new = []
        for t in range(c):
            members = np.flatnonzero(lab == t)
            if members.size == 0:                  # cannot happen (a medoid is its own nearest), kept for safety
                new.append(med[t])
                continue
            cost = D[np.ix_(members, members)].sum(axis=1)
            new.append(int(members[int(np.argmin(cost))]))
        if new == med:
            break
        med = new
    return med, assign(D, med)


def silhouette_fixed(D, lab, c):
    """floor(s_i * 2^32) for every query i (exact: integer sums and one integer division)."""
    Q = D.shape[0]
    sizes = np.bincount(lab, minlength=c)
    out = np.zeros(Q, dtype=object)
    for i in range(Q):
        A = int(lab[i])
        if sizes[A] <= 1:
            out[i] = 0
            continue
        sums = np.bincount(lab, weights=D[i], minlength=c).astype(np.int64)
        SA, na = int(sums[A]), int(sizes[A]) - 1           # D[i][i] = 0 is in the sum
        best = None
        for B in range(c):
            if B == A or sizes[B] == 0:
                continue
            SB, nb = int(sums[B]), int(sizes[B])
            if best is None or SB * best[1] < best[0] * nb:
                best = (SB, nb)
        if best is None:
            out[i] = 0
            continue
        SB, nb = best
        N = SB * na - SA * nb                              # (b - a) * na * nb
        M = max(SA * nb, SB * na)                          # max(a, b) * na * nb
        out[i] = 0 if M == 0 else (N * SCALE) // M         # floor division, also for N < 0
    return out


def cluster_batch(q_strings, c_min=2, c_max=8):
    """Clusterings for every c in [c_min, c_max] (c <= Q - 1): scores, the chosen c, its medoids and labels."""
    D = pair_distances(q_strings)
    Q = D.shape[0]
    c_hi = min(c_max, Q - 1)
    scores, runs = {}, {}
    for c in range(c_min, c_hi + 1):
        med, lab = kmedoids(D, c)
        scores[c] = int(sum(silhouette_fixed(D, lab, c)))
        runs[c] = (med, lab)
    if not scores:
        return {"c": 1, "medoids": [int(np.argmin(D.sum(axis=1)))] if Q else [], "labels": np.zeros(Q, np.int64),
                "scores": {}}
    best = max(scores, key=lambda cc: (scores[cc], -cc))
    med, lab = runs[best]
    return {"c": best, "medoids": med, "labels": lab, "scores": scores}
