"""Seeded synthetic MACCS-166-like inputs (shared by the oracle side and the CUDA side).

This module only *makes inputs*: libraries, queries, k mixes and arrival times.
It holds none of the search method's arithmetic, so both the oracle and the
CUDA path can take their inputs from it without sharing any method code.

The recipe stands in for the paper's PubChem MACCS-166 library (Sec. 4.1-4.2,
~95.4 M molecules, 166 keys): bit j of a record ~ Bernoulli(p_j) with
p_j ~ Beta(0.5, 2) drawn once from a chemistry seed, bit 0 always 0, and 1 %
planted near-duplicates (a copy of an earlier record with 1-5 bits flipped).
The implementation is ``fps_synth.c`` (counter-based SplitMix64 draws, so the
result does not depend on the thread count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fps_synth.c")
_SO = os.path.join(_HERE, "libfps_synth.so")
_lock = threading.Lock()
_lib = None

BITS = 166
WORDS = 3
LINE_BYTES = BITS + 1          # 166 characters + '\n'


def build(force: bool = False) -> str:
    """Compile the generator with gcc (portable C, no arch-specific flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u64, i32 = ctypes.c_uint64, ctypes.c_int
            vp = ctypes.c_void_p
            lib.synth_thresholds.argtypes = [u64, vp, vp]
            lib.synth_planted.argtypes = [u64, u64, vp, vp, vp]
            lib.synth_planted.restype = i32
            lib.synth_packed.argtypes = [u64, u64, u64, u64, i32, vp]
            lib.synth_text.argtypes = [u64, u64, u64, u64, i32, vp]
            lib.synth_packed_at.argtypes = [u64, u64, vp, u64, vp]
            lib.synth_draw.argtypes = [u64, u64, u64]
            lib.synth_draw.restype = u64
            lib.synth_wide.argtypes = [u64, u64, u64, u64, i32, i32, vp, vp]
            lib.synth_wide.restype = i32
            lib.synth_wide_at.argtypes = [u64, u64, vp, u64, i32, vp]
            lib.synth_wide_at.restype = i32
            _lib = lib
    return _lib


def _threads(threads):
    return int(threads) if threads else max(1, os.cpu_count() or 1)


def probabilities(chem_seed: int = 0):
    """(thresholds uint32[166], p float64[166]) of the chemistry vector."""
    lib = _load()
    T = np.zeros(BITS, np.uint32)
    p = np.zeros(BITS, np.float64)
    lib.synth_thresholds(chem_seed, T.ctypes.data, p.ctypes.data)
    return T, p


def packed(n: int, seed: int, start: int = 0, chem_seed: int = 0, threads=None) -> np.ndarray:
    """Records [start, start+n) of library `seed`, as uint64[n, 3] (bit j -> word j//64, bit j%64)."""
    lib = _load()
    out = np.empty((int(n), WORDS), np.uint64)
    if n:
        lib.synth_packed(chem_seed, seed, start, int(n), _threads(threads), out.ctypes.data)
    return out


def packed_at(idx, seed: int, chem_seed: int = 0) -> np.ndarray:
    """Records of library `seed` at the given indices, uint64[len(idx), 3]."""
    lib = _load()
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    out = np.empty((idx.size, WORDS), np.uint64)
    if idx.size:
        lib.synth_packed_at(chem_seed, seed, idx.ctypes.data, idx.size, out.ctypes.data)
    return out


def text(n: int, seed: int, start: int = 0, chem_seed: int = 0, threads=None) -> bytes:
    """Records [start, start+n) as '0'/'1' text lines of 166 characters, each ending in '\\n'."""
    lib = _load()
    buf = np.empty(int(n) * LINE_BYTES, np.uint8)
    if n:
        lib.synth_text(chem_seed, seed, start, int(n), _threads(threads), buf.ctypes.data)
    return buf.tobytes()


def text_buffer(n: int, seed: int, start: int = 0, chem_seed: int = 0, threads=None) -> np.ndarray:
    """Like :func:`text` but returns the uint8 buffer itself (no copy to bytes)."""
    lib = _load()
    buf = np.empty(int(n) * LINE_BYTES, np.uint8)
    if n:
        lib.synth_text(chem_seed, seed, start, int(n), _threads(threads), buf.ctypes.data)
    return buf


def planted(seed: int, i: int):
    """(src, m, positions) if record i was planted as a near-duplicate of record src, else None."""
    lib = _load()
    src = ctypes.c_uint64(0)
    m = ctypes.c_int(0)
    pos = (ctypes.c_int * 5)()
    if not lib.synth_planted(seed, i, ctypes.byref(src), ctypes.byref(m), pos):
        return None
    return int(src.value), int(m.value), [int(pos[a]) for a in range(m.value)]


def draw(seed: int, rec: int, slot: int) -> int:
    """One raw uniform 64-bit draw (SplitMix64, counter = (rec, slot))."""
    return int(_load().synth_draw(seed, rec, slot))


def packed_to_strings(words: np.ndarray) -> list:
    """Format packed records as 166-character '0'/'1' strings (character j = word j//64, bit j%64)."""
    words = np.asarray(words, dtype=np.uint64).reshape(-1, WORDS)
    bits = np.unpackbits(words.view(np.uint8).reshape(-1, WORDS * 8), axis=1, bitorder="little")
    return [row[:BITS].tobytes().translate(bytes.maketrans(b"\x00\x01", b"01")).decode()
            for row in bits]


def strings_to_text(rows, cids=None, sep: str = " ", crlf: bool = False) -> bytes:
    """Join fingerprint strings into library text (optionally '<cid><sep><bits>' lines)."""
    eol = "\r\n" if crlf else "\n"
    if cids is None:
        return "".join(r + eol for r in rows).encode()
    return "".join(f"{c}{sep}{r}{eol}" for c, r in zip(cids, rows)).encode()


def k_mix(q: int, seed: int = 2, choices=(1, 10, 30, 100, 1000)) -> np.ndarray:
    """Per-query k drawn uniformly from `choices` (the mixed-k batch workload)."""
    return np.array([choices[draw(seed, i, 7) % len(choices)] for i in range(q)], np.int32)


def query_seed(config_id: int) -> int:
    """Seed of the generated query set for workload `config_id` (1000 + id)."""
    return 1000 + int(config_id)


# ------------------------------------------------------------------ wide
def wide_words(n_bits: int) -> int:
    return (int(n_bits) + 63) // 64


def wide_packed(n: int, n_bits: int, seed: int, start: int = 0, chem_seed: int = 0, threads=None) -> np.ndarray:
    """Records [start, start+n) of a wide library (n_bits per record): uint64 [n, W], bits past n_bits zero."""
    out = np.zeros((int(n), wide_words(n_bits)), np.uint64)
    if _load().synth_wide(chem_seed, seed, start, int(n), int(n_bits), _threads(threads), out.ctypes.data, None):
        raise ValueError("n_bits must be in 1..4096")
    return out


def wide_text(n: int, n_bits: int, seed: int, start: int = 0, chem_seed: int = 0, threads=None) -> bytes:
    """The same records as n lines of n_bits '0'/'1' characters plus '\n'."""
    buf = ctypes.create_string_buffer(int(n) * (int(n_bits) + 1))
    if _load().synth_wide(chem_seed, seed, start, int(n), int(n_bits), _threads(threads), None, buf):
        raise ValueError("n_bits must be in 1..4096")
    return buf.raw


def wide_at(idx, n_bits: int, seed: int, chem_seed: int = 0) -> np.ndarray:
    """Wide records chosen by index (e.g. queries that are library members)."""
    idx = np.ascontiguousarray(np.asarray(idx, np.uint64).reshape(-1))
    out = np.zeros((idx.size, wide_words(n_bits)), np.uint64)
    if _load().synth_wide_at(chem_seed, seed, idx.ctypes.data, idx.size, int(n_bits), out.ctypes.data):
        raise ValueError("n_bits must be in 1..4096")
    return out


def wide_to_strings(words: np.ndarray, n_bits: int) -> list:
    """Format packed wide records as n_bits-character '0'/'1' strings (character j = word j//64, bit j%64)."""
    W = wide_words(n_bits)
    words = np.asarray(words, dtype=np.uint64).reshape(-1, W)
    bits = np.unpackbits(words.view(np.uint8).reshape(-1, W * 8), axis=1, bitorder="little")[:, :n_bits]
    return ["".join("1" if b else "0" for b in row) for row in bits]
