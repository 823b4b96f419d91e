"""Golden fixtures (hand-derived closed forms; oracle-written seeded results) and generator checks."""
import os

import numpy as np

import oracle
import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def expand(pat):
    out = ""
    for piece in pat.split("+"):
        chars, _, rep = piece.partition("*")
        out += chars * (int(rep) if rep else 1)
    assert len(out) == 166, pat
    return out


def test_closed_form_fixture():
    rows = []
    with open(os.path.join(GOLD, "closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            q, x, d, _ = [c.strip() for c in line.split("|")]
            rows.append((expand(q), expand(x), int(d)))
    assert len(rows) >= 10
    for q, x, d in rows:
        assert oracle.distances(synth.strings_to_text([x]), q).tolist() == [d]


def test_seeded_topk_fixture():
    want = {}
    with open(os.path.join(GOLD, "topk_seed0_n20000.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            q, r, i, d = map(int, line.split())
            want.setdefault(q, []).append((i, d))
    text = synth.text(20000, 0)
    queries = synth.packed_to_strings(synth.packed(3, 1001))
    for q, pairs in want.items():
        idx, dist, _ = oracle.topk(text, queries[q], 30)
        assert list(zip(idx.tolist(), dist.tolist())) == pairs


def test_seeded_wide_fixture():
    """n-bit extension: 1024-bit top-20, Manhattan and Tanimoto (tests/golden/make_golden.py)."""
    want = {}
    with open(os.path.join(GOLD, "wide_seed21_n3000.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            m, q, r, i, a, b = map(int, line.split())
            want.setdefault((m, q), []).append((i, a, b))
    assert sorted(want) == [(0, 0), (0, 1), (1, 0), (1, 1)]
    text = synth.wide_text(3000, 1024, 21)
    queries = synth.wide_to_strings(synth.wide_packed(2, 1024, 1021), 1024)
    for (m, q), rows in want.items():
        idx, num, den = oracle.wide_topk(text, 1024, queries[q], 20, m)
        assert list(zip(idx.tolist(), num.tolist(), den.tolist())) == rows


def test_seeded_cluster_fixture():
    """Batch clustering search: scores per count, the chosen count, medoids and labels."""
    from oracle import cluster

    scores, best, med, lab = {}, None, None, None
    with open(os.path.join(GOLD, "cluster_seed1400.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "score":
                scores[int(vals[0])] = int(vals[1])
            elif key == "best":
                best = int(vals[0])
            elif key == "medoids":
                med = [int(v) for v in vals]
            elif key == "labels":
                lab = [int(v) for v in vals]
    res = cluster.cluster_batch(synth.packed_to_strings(synth.packed(120, 1400)), 2, 6)
    assert res["scores"] == scores and res["c"] == best
    assert [int(m) for m in res["medoids"]] == med and res["labels"].tolist() == lab


def test_generator_is_thread_count_independent_and_consistent():
    a = synth.packed(50000, 3, threads=1)
    b = synth.packed(50000, 3, threads=7)
    assert np.array_equal(a, b)
    c = synth.packed(1000, 3, start=20000)
    assert np.array_equal(c, a[20000:21000])
    assert np.array_equal(synth.packed_at([5, 20000, 49999], 3), a[[5, 20000, 49999]])
    t = synth.text(200, 3)
    assert t.decode().splitlines() == synth.packed_to_strings(a[:200])


def test_generator_shape_matches_recipe():
    a = synth.packed(200000, 0)
    assert np.all(a[:, 0] & np.uint64(1) == 0)                     # key 0 is never set
    assert np.all(a[:, 2] >> np.uint64(38) == 0)                   # no bits beyond key 165
    bits = np.unpackbits(a.view(np.uint8), axis=1, bitorder="little")[:, :166]
    pc = bits.sum(1)
    _, p = synth.probabilities(0)
    assert abs(pc.mean() - p.sum()) < 0.2                           # E[popc] = sum_j p_j
    assert 25 < pc.mean() < 45 and 3 < pc.std() < 7
    assert np.allclose(bits.mean(0), p, atol=0.01)
    planted = sum(synth.planted(0, i) is not None for i in range(20000))
    assert 140 <= planted <= 260                                    # ~1 %
    _, pbeta = synth.probabilities(0)
    assert abs(pbeta[1:].mean() - 0.2) < 0.05                       # Beta(0.5, 2) has mean 0.2
