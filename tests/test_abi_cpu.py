"""C ABI checks that need no GPU: the library loads, exports every declared
symbol, and its host-only helpers (query packing, text parsing) agree with the
generator's packed form and the oracle's parse rules."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fps():
    import __graft_entry__ as ge

    ge._cuda_build_module().build()
    import paper_1906_06170_gb300 as mod

    return mod


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(fps_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(fps):
    names = declared_functions()
    assert len(names) >= 10
    lib = ctypes.CDLL(fps.library_path())
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(fps):
    for st in range(10):
        assert fps._lib.fps_status_string(st)


def test_pack_query_matches_generator_bit_order(fps):
    a = synth.packed(50, 5)
    for row, s in zip(a, synth.packed_to_strings(a)):
        assert np.array_equal(fps.fps_pack_query(s), row)
    with pytest.raises(fps.FpsError):
        fps.fps_pack_query("0" * 165 + "2")


def test_pack_text_matches_generator_and_oracle_rules(fps):
    n = 3000
    a = synth.packed(n, 6)
    packed, cids = fps.fps_pack_text(synth.text(n, 6))
    assert np.array_equal(packed, a) and np.array_equal(cids, np.arange(n))
    rows = synth.packed_to_strings(a[:5])
    t = synth.strings_to_text(rows, cids=[7, 8, 11050016, 3, 9], sep="\t", crlf=True)
    packed, cids = fps.fps_pack_text(t)
    assert np.array_equal(packed, a[:5]) and cids.tolist() == [7, 8, 11050016, 3, 9]
    assert cids.tolist() == oracle.cids(t).tolist()
    bad = synth.strings_to_text([rows[0], rows[1], rows[2][:-1] + "x"])
    with pytest.raises(fps.FpsError) as e:
        fps.fps_pack_text(bad)
    with pytest.raises(oracle.OracleError) as eo:
        oracle.count(bad)
    assert e.value.line == eo.value.line == 3
    long = synth.strings_to_text(["0" + r for r in rows])
    with pytest.raises(fps.FpsError):
        fps.fps_pack_text(long)
    packed, _ = fps.fps_pack_text(long, fps.FPS_LOAD_ACCEPT_167)
    assert np.array_equal(packed, a[:5])


def test_pack_text_large_parallel_parse(fps):
    n = 20000          # > 1 MiB of text: the multi-threaded parse path
    text = synth.text(n, 9)
    packed, _ = fps.fps_pack_text(text)
    assert np.array_equal(packed, synth.packed(n, 9))
    lines = text.split(b"\n")
    lines[12345] = lines[12345][:-1]
    with pytest.raises(fps.FpsError) as e:
        fps.fps_pack_text(b"\n".join(lines))
    assert e.value.line == 12346
