"""CPU oracle for FPScreen's search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The CUDA search path neither
imports it nor shares any code with it; the two meet only in the seeded input
generator (``synth``), which holds none of the method's arithmetic.

Two independent restatements of the paper's search (Sec. 4.3 and Fig. 3):

* :func:`topk` and friends -- the plain C oracle in ``fps_oracle.c``: parse the
  '0'/'1' library text, compare characters, fully sort (distance, index) pairs.
* :func:`fig3_topk` -- NumPy, literally the six steps of Fig. 3: matrix A,
  vector b, broadcast C = A - b, K = row sums of |C|, pair with the row
  number, stable ascending sort, first k.

Ties in distance are ordered by ascending 0-based line index (the paper does
not say; this reading makes the answer unique).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fps_oracle.c")
_SO = os.path.join(_HERE, "libfps_oracle.so")
_lock = threading.Lock()
_lib = None

BITS = 166
ACCEPT_167 = 1
OK, ERR_ARG, ERR_PARSE, ERR_NOMEM = 0, 1, 3, 9


class OracleError(RuntimeError):
    def __init__(self, status, line=0):
        super().__init__(f"oracle status {status}" + (f" at line {line}" if line else ""))
        self.status = status
        self.line = line


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable C, -O2, pthreads)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, sz, i64, i32, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int, ctypes.c_uint
            lib.oracle_count.argtypes = [vp, sz, u32, vp, vp]
            lib.oracle_distances.argtypes = [vp, sz, u32, ctypes.c_char_p, i32, vp, i64, vp, vp]
            lib.oracle_cids.argtypes = [vp, sz, u32, vp, i64, vp, vp]
            lib.oracle_topk.argtypes = [vp, sz, u32, ctypes.c_char_p, i64, i32, vp, vp, vp, vp, vp]
            lib.oracle_topk_many.argtypes = [vp, sz, u32, ctypes.c_char_p, i64, vp, vp, i32, vp, vp, vp, vp]
            lib.oracle_combine.argtypes = [vp, vp, i64, i64, vp, vp, vp]
            lib.oracle_wide_topk.argtypes = [vp, sz, i32, ctypes.c_char_p, i64, i32, i32, vp, vp, vp, vp, vp]
            for f in (lib.oracle_count, lib.oracle_distances, lib.oracle_cids, lib.oracle_topk,
                      lib.oracle_topk_many, lib.oracle_combine):
                f.restype = i32
            _lib = lib
    return _lib


def _buf(text):
    """(pointer, length, keepalive) for bytes / bytearray / uint8 ndarray text."""
    if isinstance(text, np.ndarray):
        a = np.ascontiguousarray(text, dtype=np.uint8)
        return a.ctypes.data, a.size, a
    b = bytes(text)
    cb = ctypes.create_string_buffer(b, len(b))
    return ctypes.addressof(cb), len(b), cb


def _threads(threads):
    return int(threads) if threads else max(1, os.cpu_count() or 1)


def _q(query: str) -> bytes:
    q = query.encode() if isinstance(query, str) else bytes(query)
    if len(q) != BITS:
        raise ValueError("query must have 166 characters")
    return q


def count(text, flags: int = 0) -> int:
    lib = _load()
    p, n, keep = _buf(text)
    out, err = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.oracle_count(p, n, flags, ctypes.byref(out), ctypes.byref(err))
    if st:
        raise OracleError(st, err.value)
    return out.value


def distances(text, query: str, flags: int = 0, threads=None) -> np.ndarray:
    """K_i = sum_j |A_ij - b_j| for every library row (Sec. 4.3; Fig. 3 steps 3-4)."""
    lib = _load()
    p, n, keep = _buf(text)
    cap = count(text, flags)
    d = np.zeros(max(cap, 1), np.int32)
    out, err = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.oracle_distances(p, n, flags, _q(query), _threads(threads), d.ctypes.data, cap,
                              ctypes.byref(out), ctypes.byref(err))
    if st:
        raise OracleError(st, err.value)
    return d[: out.value]


def cids(text, flags: int = 0) -> np.ndarray:
    lib = _load()
    p, n, keep = _buf(text)
    cap = count(text, flags)
    c = np.zeros(max(cap, 1), np.int64)
    out, err = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.oracle_cids(p, n, flags, c.ctypes.data, cap, ctypes.byref(out), ctypes.byref(err))
    if st:
        raise OracleError(st, err.value)
    return c[: out.value]


def topk(text, query: str, k: int, flags: int = 0, threads=None):
    """(index int32[m], distance int32[m], cid int64[m]) with m = min(k, N): Fig. 3 steps 1-6."""
    lib = _load()
    p, n, keep = _buf(text)
    cap = max(int(k), 0)
    idx = np.zeros(max(cap, 1), np.int32)
    dist = np.zeros(max(cap, 1), np.int32)
    cid = np.zeros(max(cap, 1), np.int64)
    out, err = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.oracle_topk(p, n, flags, _q(query), int(k), _threads(threads), idx.ctypes.data, dist.ctypes.data,
                         cid.ctypes.data, ctypes.byref(out), ctypes.byref(err))
    if st:
        raise OracleError(st, err.value)
    m = out.value
    return idx[:m], dist[:m], cid[:m]


def topk_many(text, queries, ks, flags: int = 0, threads=None):
    """Per-query results [(index, distance)] for many queries against one library."""
    lib = _load()
    p, n, keep = _buf(text)
    Q = len(queries)
    ks = np.asarray(ks, dtype=np.int64).reshape(-1)
    if ks.size == 1 and Q > 1:
        ks = np.full(Q, ks[0], np.int64)
    off = np.zeros(Q + 1, np.int64)
    off[1:] = np.cumsum(np.maximum(ks, 0))
    qbuf = b"".join(_q(q) for q in queries)
    idx = np.zeros(max(int(off[-1]), 1), np.int32)
    dist = np.zeros(max(int(off[-1]), 1), np.int32)
    nout = np.zeros(max(Q, 1), np.int64)
    err = ctypes.c_int64(0)
    st = lib.oracle_topk_many(p, n, flags, qbuf, Q, ks.ctypes.data, off.ctypes.data, _threads(threads),
                              idx.ctypes.data, dist.ctypes.data, nout.ctypes.data, ctypes.byref(err))
    if st:
        raise OracleError(st, err.value)
    return [(idx[off[q]: off[q] + nout[q]].copy(), dist[off[q]: off[q] + nout[q]].copy()) for q in range(Q)]


def combine(parts, k: int):
    """"Combined and sorted" (text after Fig. 3): merge (index, distance) lists by re-sorting."""
    lib = _load()
    idx = np.ascontiguousarray(np.concatenate([np.asarray(a, np.int32) for a, _ in parts] or [np.zeros(0, np.int32)]))
    dist = np.ascontiguousarray(np.concatenate([np.asarray(b, np.int32) for _, b in parts] or [np.zeros(0, np.int32)]))
    oi = np.zeros(max(k, 1), np.int32)
    od = np.zeros(max(k, 1), np.int32)
    out = ctypes.c_int64(0)
    st = lib.oracle_combine(idx.ctypes.data, dist.ctypes.data, idx.size, int(k), oi.ctypes.data, od.ctypes.data,
                            ctypes.byref(out))
    if st:
        raise OracleError(st)
    return oi[: out.value], od[: out.value]


def fig3_topk(rows, query: str, k: int):
    """NumPy restatement of Fig. 3, step by step (small inputs only).

    1) A = library fingerprints as an N x 166 matrix of 0/1 (row i = line i);
    2) b = the target's 166-vector;
    3) C_ij = A_ij - b_j by broadcasting;
    4) K = row sums of |C| (the Manhattan distance of Sec. 4.3);
    5) pair K with the row number;
    6) sort ascending (stable, so equal K keep row order) and take the first k.
    """
    A = np.array([[int(c) for c in r] for r in rows], dtype=np.int64).reshape(-1, BITS)
    b = np.array([int(c) for c in query], dtype=np.int64)
    C = A - b
    K = np.abs(C).sum(axis=1)
    order = np.argsort(K, kind="stable")[: max(int(k), 0)]
    return order.astype(np.int32), K[order].astype(np.int32)


# ------------------------------------------------------------------ wide
MANHATTAN, TANIMOTO = 0, 1


def wide_topk(text, n_bits: int, query: str, k: int, metric: int = MANHATTAN, threads=None):
    """Top-k rows of a wide library (lines of n_bits '0'/'1' characters).

    Manhattan: ascending d = number of differing characters; Tanimoto: descending c / u
    (c = both '1', u = either '1'; 1 when u = 0), compared exactly.  Ties: ascending row.
    Returns (rows, num, den): Manhattan num = d, den = 1; Tanimoto num = c, den = u."""
    lib = _load()
    p, n, keep = _buf(text)
    q = query.encode() if isinstance(query, str) else bytes(query)
    if len(q) != n_bits:
        raise OracleError(ERR_ARG)
    m = max(int(k), 1)
    idx, num, den = np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m, np.int32)
    out, err = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.oracle_wide_topk(p, n, int(n_bits), q, int(k), int(metric), _threads(threads), idx.ctypes.data,
                              num.ctypes.data, den.ctypes.data, ctypes.byref(out), ctypes.byref(err))
    if st:
        raise OracleError(st, err.value)
    c = out.value
    return idx[:c], num[:c], den[:c]
