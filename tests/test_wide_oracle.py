"""Pins of the wide-fingerprint / Tanimoto oracle (oracle.wide_topk) against definitions that do not use it:
Python-integer brute force with exact fractions, closed forms, symmetry, the triangle inequality of the
Jaccard distance 1 - Tanimoto, and the 166-bit oracle at n = 166."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def brute(rows, q, k, metric):
    qi = int(q[::-1], 2)
    keyed = []
    for i, r in enumerate(rows):
        x = int(r[::-1], 2)
        if metric == oracle.MANHATTAN:
            keyed.append(((bin(qi ^ x).count("1"),), i, bin(qi ^ x).count("1"), 1))
        else:
            c, u = bin(qi & x).count("1"), bin(qi | x).count("1")
            s = Fraction(c, u) if u else Fraction(1)
            keyed.append(((-s,), i, c, u))
    keyed.sort(key=lambda t: (t[0], t[1]))
    top = keyed[:k]
    return [t[1] for t in top], [t[2] for t in top], [t[3] for t in top]


def text_of(rows):
    return ("\n".join(rows) + "\n").encode() if rows else b""


@pytest.mark.parametrize("n_bits", [1, 7, 64, 65, 130, 512])
@pytest.mark.parametrize("metric", [0, 1])
def test_wide_oracle_equals_brute_force(n_bits, metric):
    rng = np.random.default_rng(n_bits * 10 + metric)
    for trial in range(4):
        n = int(rng.integers(1, 300))
        dens = rng.uniform(0.02, 0.6)
        rows = ["".join("1" if v else "0" for v in rng.random(n_bits) < dens) for _ in range(n)]
        rows += rows[: n // 5]                                   # duplicates: ties broken by row
        q = rows[int(rng.integers(0, len(rows)))] if trial % 2 else \
            "".join("1" if v else "0" for v in rng.random(n_bits) < dens)
        for k in (1, 5, len(rows), len(rows) + 3):
            wi, wn, wd = brute(rows, q, k, metric)
            gi, gn, gd = oracle.wide_topk(text_of(rows), n_bits, q, k, metric)
            assert gi.tolist() == wi and gn.tolist() == wn and gd.tolist() == wd, (n_bits, metric, trial, k)


def test_tanimoto_closed_forms():
    n_bits = 200
    ones = "1" * n_bits
    zeros = "0" * n_bits
    half_a = "1" * 100 + "0" * 100
    half_b = "0" * 100 + "1" * 100
    sub = "1" * 40 + "0" * 160                                   # subset of half_a
    rows = [zeros, half_a, half_b, sub, ones]
    t = text_of(rows)
    i, c, u = oracle.wide_topk(t, n_bits, half_a, 5, oracle.TANIMOTO)
    sims = {int(r): (int(a), int(b)) for r, a, b in zip(i, c, u)}
    assert sims[1] == (100, 100)                                 # identical: 1
    assert sims[2] == (0, 200)                                   # disjoint: 0
    assert sims[3] == (40, 100)                                  # subset: popc(sub) / popc(half_a)
    assert sims[4] == (100, 200)                                 # superset ones: 100 / 200
    assert sims[0] == (0, 100)
    assert i.tolist() == [1, 4, 3, 0, 2] or i.tolist() == [1, 4, 3, 2, 0]
    assert i.tolist()[-2:] == [0, 2]                             # 0/100 and 0/200 tie at 0: row order
    i, c, u = oracle.wide_topk(t, n_bits, zeros, 5, oracle.TANIMOTO)
    assert i[0] == 0 and (c[0], u[0]) == (0, 0)                  # two empty sets: similarity 1, first
    i, d, _ = oracle.wide_topk(t, n_bits, ones, 5, oracle.MANHATTAN)
    assert dict(zip(i.tolist(), d.tolist()))[0] == n_bits       # complement: every character differs


def pair(a, b, n_bits, metric):
    _, num, den = oracle.wide_topk(text_of([b]), n_bits, a, 1, metric)
    return int(num[0]), int(den[0])


def test_symmetry_and_jaccard_triangle_inequality():
    n_bits = 96
    rng = np.random.default_rng(7)
    rows = ["".join("1" if v else "0" for v in rng.random(n_bits) < rng.uniform(0.05, 0.5)) for _ in range(24)]

    def jdist(a, b):
        c, u = pair(a, b, n_bits, oracle.TANIMOTO)
        return 1 - (Fraction(c, u) if u else Fraction(1))

    for _ in range(60):
        a, b, c = (rows[int(j)] for j in rng.integers(0, len(rows), 3))
        assert pair(a, b, n_bits, oracle.TANIMOTO) == pair(b, a, n_bits, oracle.TANIMOTO)
        assert pair(a, b, n_bits, oracle.MANHATTAN) == pair(b, a, n_bits, oracle.MANHATTAN)
        assert jdist(a, c) <= jdist(a, b) + jdist(b, c)
        da, db = pair(a, c, n_bits, oracle.MANHATTAN)[0], pair(a, b, n_bits, oracle.MANHATTAN)[0]
        assert da <= db + pair(b, c, n_bits, oracle.MANHATTAN)[0]


def test_wide_manhattan_at_166_bits_equals_the_maccs_oracle():
    text = synth.text(5000, 71)
    for q in synth.packed_to_strings(synth.packed(3, 1071)):
        wi, wd, _ = oracle.topk(text, q, 100)
        gi, gn, gdn = oracle.wide_topk(text, 166, q, 100, oracle.MANHATTAN)
        assert gi.tolist() == wi.tolist() and gn.tolist() == wd.tolist() and set(gdn.tolist()) == {1}


def test_wide_generator_text_round_trip_and_parse_errors():
    t = synth.wide_text(50, 300, 9)
    rows = synth.wide_to_strings(synth.wide_packed(50, 300, 9), 300)
    assert t == text_of(rows)
    gi, _, _ = oracle.wide_topk(t.replace(b"\n", b"\r\n"), 300, rows[3], 1)
    assert gi.tolist() == [3]
    bad = text_of(rows[:10] + [rows[10][:-1]] + rows[11:])
    with pytest.raises(oracle.OracleError) as e:
        oracle.wide_topk(bad, 300, rows[0], 5)
    assert e.value.status == oracle.ERR_PARSE and e.value.line == 11
