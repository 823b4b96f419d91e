"""Pins for the CPU oracle, against facts fixed by the paper and by mathematics.

The oracle restates Sec. 4.3 (Manhattan distance over the 166 MACCS keys) and
Fig. 3 (pair every row with its distance, sort ascending, take the first k).
Nothing here retypes the oracle's formula: each test checks it against
something else -- Python integer XOR/bit counts, closed forms, metric
invariants, an exhaustive table, planted near-duplicates whose distance is
known by construction, textbook sorting/selection routines, and the literal
NumPy restatement of Fig. 3.
"""
import heapq
import random

import numpy as np
import pytest

import oracle
import synth

B = 166


def rand_rows(rng, n, p=0.2):
    return ["".join("1" if rng.random() < p else "0" for _ in range(B)) for _ in range(n)]


def text_of(rows):
    return synth.strings_to_text(rows)


def xor_count(a, b):
    return (int(a, 2) ^ int(b, 2)).bit_count()


@pytest.mark.parametrize("p", [0.05, 0.2, 0.5, 0.9])
def test_distance_equals_integer_xor_bitcount(p):
    rng = random.Random(int(p * 100))
    rows = rand_rows(rng, 64, p)
    for q in rand_rows(rng, 4, p):
        d = oracle.distances(text_of(rows), q)
        assert list(d) == [xor_count(q, r) for r in rows]


def test_distance_sensitive_to_every_key_position():
    # A single differing key at each position j (including the first and the last) gives 1.
    zero = "0" * B
    rows = [zero[:j] + "1" + zero[j + 1:] for j in range(B)]
    d = oracle.distances(text_of(rows), zero)
    assert list(d) == [1] * B


def test_closed_forms_all_zeros_all_ones_complement():
    rows = synth.packed_to_strings(synth.packed(300, 0))
    t = text_of(rows)
    # Fig. 1's default query is all zeros: the distance is then the number of set keys.
    assert list(oracle.distances(t, "0" * B)) == [r.count("1") for r in rows]
    assert list(oracle.distances(t, "1" * B)) == [B - r.count("1") for r in rows]
    q = synth.packed_to_strings(synth.packed(1, 1001))[0]
    qc = "".join("1" if c == "0" else "0" for c in q)
    d = oracle.distances(t, q)
    dc = oracle.distances(t, qc)
    assert np.array_equal(d + dc, np.full(len(rows), B))


def test_metric_invariants():
    rng = random.Random(7)
    rows = rand_rows(rng, 40, 0.3)
    t = text_of(rows)
    D = np.stack([oracle.distances(t, r) for r in rows])
    assert np.all(np.diag(D) == 0)                       # d(x, x) = 0
    assert np.array_equal(D, D.T)                        # symmetry
    assert D.min() >= 0 and D.max() <= B                 # 0 <= d <= 166
    for b in range(len(rows)):                           # d(a, c) <= d(a, b) + d(b, c)
        assert np.all(D <= D[:, [b]] + D[[b], :])
    for a in range(len(rows)):                           # d = |a| + |b| - 2|a AND b|
        for b in range(len(rows)):
            ia, ib = int(rows[a], 2), int(rows[b], 2)
            assert D[a, b] == ia.bit_count() + ib.bit_count() - 2 * (ia & ib).bit_count()


def test_exhaustive_low_ten_keys():
    # Every pattern of the first 10 keys (rest zero) against every other: a 1024 x 1024 table.
    rows = [format(v, "010b") + "0" * (B - 10) for v in range(1024)]
    t = text_of(rows)
    table = np.array([[bin(a ^ b).count("1") for b in range(1024)] for a in range(0, 1024, 37)])
    got = np.stack([oracle.distances(t, rows[a]) for a in range(0, 1024, 37)])
    assert np.array_equal(got, table)


def test_planted_near_duplicates_have_their_flip_count():
    n = 6000
    packed = synth.packed(n, 0)
    rows = synth.packed_to_strings(packed)
    t = text_of(rows)
    found = 0
    for i in range(n):
        info = synth.planted(0, i)
        if info is None:
            continue
        src, m, pos = info
        found += 1
        assert xor_count(rows[src], rows[i]) == m          # independent of the oracle
        d = oracle.distances(t, rows[src])
        assert d[i] == m and d[src] == 0
        idx, dist, _ = oracle.topk(t, rows[src], 60)
        assert (src, 0) in set(zip(idx.tolist(), dist.tolist()))   # the query itself comes back at 0
        if m < dist[-1]:                                    # every record closer than the 60th is listed
            assert i in set(idx.tolist())
    assert 30 <= found <= 100                               # ~1 % of records


@pytest.mark.parametrize("k", [0, 1, 5, 30, 64, 200])
def test_topk_matches_textbook_selection(k):
    rng = random.Random(k)
    rows = rand_rows(rng, 150, 0.1)          # low density: many ties
    q = rand_rows(rng, 1, 0.1)[0]
    d = [xor_count(q, r) for r in rows]
    want = sorted(range(len(rows)), key=lambda i: (d[i], i))[:k]
    want_heap = [i for _, i in heapq.nsmallest(k, [(d[i], i) for i in range(len(rows))])]
    idx, dist, cid = oracle.topk(text_of(rows), q, k)
    assert idx.tolist() == want == want_heap
    assert dist.tolist() == [d[i] for i in want]
    assert cid.tolist() == want                             # no CID column: CID = line index
    fi, fd = oracle.fig3_topk(rows, q, k)
    assert fi.tolist() == want and fd.tolist() == [d[i] for i in want]


def test_adversarial_ties():
    q = synth.packed_to_strings(synth.packed(1, 1001))[0]
    x = synth.packed_to_strings(synth.packed(2, 0))
    same = [x[0]] * 100
    idx, dist, _ = oracle.topk(text_of(same), q, 30)
    assert idx.tolist() == list(range(30)) and set(dist.tolist()) == {xor_count(q, x[0])}
    two = [x[i % 2] for i in range(101)]
    d0, d1 = xor_count(q, x[0]), xor_count(q, x[1])
    idx, dist, _ = oracle.topk(text_of(two), q, 70)
    lo = 0 if (d0, 0) < (d1, 1) else 1
    want = [i for i in range(101) if i % 2 == lo] + [i for i in range(101) if i % 2 != lo]
    assert idx.tolist() == want[:70]
    idx, dist, _ = oracle.topk(text_of(x), q, 30)           # N < k
    assert len(idx) == 2
    idx, dist, _ = oracle.topk(text_of(same[:30]), q, 30)   # k = N
    assert idx.tolist() == list(range(30))
    idx, dist, _ = oracle.topk(b"", q, 30)                  # empty library
    assert len(idx) == 0


def test_parse_formats_and_errors():
    r = synth.packed_to_strings(synth.packed(3, 0))
    q = r[1]
    for sep in (" ", "\t", ","):
        t = synth.strings_to_text(r, cids=[11050016, 11092947, 89257755], sep=sep)
        idx, dist, cid = oracle.topk(t, q, 3)
        assert idx[0] == 1 and dist[0] == 0 and cid[0] == 11092947
    t = synth.strings_to_text(r, crlf=True)
    assert oracle.count(t) == 3
    assert oracle.count(t[:-1]) == 3                        # no final newline
    assert oracle.count(t[:-2]) == 3
    bad = synth.strings_to_text([r[0], r[1][:-1] + "2", r[2]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.count(bad)
    assert e.value.line == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.count(synth.strings_to_text([r[0], r[1][:-1], r[2]]))
    assert e.value.line == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.count(synth.strings_to_text([r[0], "", r[2]]))
    assert e.value.line == 2
    long = synth.strings_to_text(["0" + x for x in r])
    with pytest.raises(oracle.OracleError):
        oracle.count(long)
    assert oracle.count(long, oracle.ACCEPT_167) == 3
    assert list(oracle.distances(long, r[0], oracle.ACCEPT_167)) == [xor_count(r[0], x) for x in r]
    with pytest.raises(oracle.OracleError):
        oracle.count(synth.strings_to_text(["1" + x for x in r]), oracle.ACCEPT_167)


def test_combined_and_sorted_shards():
    # The text after Fig. 3: strides searched separately, their lists merged and re-sorted.
    n = 3000
    rows = synth.packed_to_strings(synth.packed(n, 0))
    q = synth.packed_to_strings(synth.packed(1, 1001))[0]
    whole = oracle.topk(text_of(rows), q, 40)
    parts = []
    for lo, hi in ((0, 1000), (1000, 2100), (2100, n)):
        i, d, _ = oracle.topk(text_of(rows[lo:hi]), q, 40)
        parts.append((i + lo, d))
    ci, cd = oracle.combine(parts, 40)
    assert ci.tolist() == whole[0].tolist() and cd.tolist() == whole[1].tolist()


def test_topk_many_equals_single_calls():
    rows = synth.packed_to_strings(synth.packed(2000, 0))
    qs = synth.packed_to_strings(synth.packed(5, 1002))
    ks = [1, 10, 30, 100, 0]
    many = oracle.topk_many(text_of(rows), qs, ks)
    for q, k, (i, d) in zip(qs, ks, many):
        i1, d1, _ = oracle.topk(text_of(rows), q, k)
        assert i.tolist() == i1.tolist() and d.tolist() == d1.tolist()
