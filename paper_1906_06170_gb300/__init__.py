"""Python binding of the FPScreen GB300 search library (C ABI in include/fps.h).

Argument marshalling only: every step of a search runs in the CUDA kernels of
``libfps.so``.  The names mirror the C entry points.  Host inputs are NumPy
arrays; device inputs/outputs are ``torch`` CUDA tensors (PyTorch supplies
device memory and streams).  If ``libfps.so`` has not been built the import
fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libfps.so")

FPS_BITS, FPS_WORDS, FPS_K_MAX, FPS_NOALLOC_K_MAX = 166, 3, 1920, 128
(FPS_OK, FPS_ERR_INVALID_ARG, FPS_ERR_IO, FPS_ERR_PARSE, FPS_ERR_BUDGET, FPS_ERR_CUDA, FPS_ERR_TIMEOUT,
 FPS_ERR_OVERFLOW_INTERNAL, FPS_ERR_UNSUPPORTED, FPS_ERR_NOMEM) = range(10)
FPS_LOAD_ACCEPT_167, FPS_LOAD_NO_BUCKETS, FPS_LOAD_TC_OPERAND, FPS_LOAD_TC_INT8 = 0x1, 0x2, 0x4, 0x8
FPS_LOAD_TC_FP4 = 0x10
(FPS_PATH_AUTO, FPS_PATH_POPC, FPS_PATH_POPC_BATCH, FPS_PATH_TC_FP8, FPS_PATH_TC_I8,
 FPS_PATH_LEARNED, FPS_PATH_TC_FP4) = range(7)
FPS_TUNE_CLASS_LEN = 32
FPS_SEARCH_DEVICE_IO = 0x1

if not os.path.exists(_SO):
    raise ImportError(f"{_SO} is missing: build the CUDA library first (__graft_entry__.build())")
_lib = ctypes.CDLL(_SO)


class FpsError(RuntimeError):
    def __init__(self, status: int, where: str = "", line: int = 0):
        msg = _lib.fps_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})" + (f" at line {line}" if line else ""))
        self.status = status
        self.line = line


class fps_load_desc(ctypes.Structure):
    _fields_ = [("path", ctypes.c_char_p), ("text", ctypes.c_void_p), ("text_len", ctypes.c_size_t),
                ("packed", ctypes.c_void_p), ("n_packed", ctypes.c_size_t), ("cids", ctypes.c_void_p),
                ("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t), ("flags", ctypes.c_uint32),
                ("err_line", ctypes.POINTER(ctypes.c_size_t))]


class fps_library_info(ctypes.Structure):
    _fields_ = [("n_records", ctypes.c_int64), ("n_tiles", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("device", ctypes.c_int), ("bucketed", ctypes.c_int), ("has_tc_operand", ctypes.c_int),
                ("bucket_count", ctypes.c_int64 * (FPS_BITS + 1)), ("has_tc_fp4", ctypes.c_int)]


class fps_search_stats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_int64), ("fallbacks", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("path_used", ctypes.c_int64), ("device_fallbacks", ctypes.c_int64), ("tile_param", ctypes.c_int64)]


class fps_search_opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("flags", ctypes.c_uint32), ("timeout_s", ctypes.c_double),
                ("stats", ctypes.POINTER(fps_search_stats)), ("tau", ctypes.c_void_p)]


_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
_lib.fps_status_string.argtypes = [_i32]
_lib.fps_status_string.restype = ctypes.c_char_p
_lib.fps_library_load.argtypes = [ctypes.POINTER(fps_load_desc), ctypes.POINTER(_vp)]
_lib.fps_release.argtypes = [_vp]
_lib.fps_library_info_get.argtypes = [_vp, ctypes.POINTER(fps_library_info)]
_lib.fps_library_cid.argtypes = [_vp, _i64, ctypes.POINTER(_i64)]
_lib.fps_search.argtypes = [_vp, ctypes.c_char_p, _i32, _vp, _vp, _vp, ctypes.POINTER(_i32), _vp]
_lib.fps_search_packed.argtypes = [_vp, _vp, _i32, _vp, _vp, _vp, ctypes.POINTER(fps_search_opts), _vp]
_lib.fps_search_batch.argtypes = [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(fps_search_opts), _vp]
_lib.fps_sync.argtypes = [_vp, _vp]
_lib.fps_search_noalloc.argtypes = [_vp, _vp, _i32, _vp, _vp, _vp, _vp]
_lib.fps_merge_topk.argtypes = [_vp, _vp, _vp, _i32, _i32, _vp, _vp, ctypes.POINTER(_i32)]
_lib.fps_wide_load.argtypes = [_vp, ctypes.c_size_t, _vp, ctypes.c_size_t, _i32, _i32, ctypes.c_size_t,
                               ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t)]
_lib.fps_wide_info.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_size_t)]
_lib.fps_wide_search.argtypes = [_vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, ctypes.c_uint32, _vp]
_lib.fps_wide_release.argtypes = [_vp]
_lib.fps_cluster_search.argtypes = [_vp, _vp, _i32, _i32, _i32, _i32, ctypes.POINTER(_i32), _vp, _vp, _vp, _vp, _vp,
                                    _vp, _vp]
_lib.fps_search_shards.argtypes = [_vp, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp,
                                   ctypes.POINTER(fps_search_opts), _vp, _vp]
_lib.fps_batch_plan_create.argtypes = [_vp, _i32, _vp, _i32, _i32, ctypes.POINTER(_vp)]
_lib.fps_batch_plan_run.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(fps_search_stats), _vp]
_lib.fps_batch_plan_release.argtypes = [_vp]
_lib.fps_mlp_param_count.restype = ctypes.c_size_t
_lib.fps_mlp_create.argtypes = [_i32, ctypes.POINTER(_vp)]
_lib.fps_mlp_release.argtypes = [_vp]
_lib.fps_mlp_set_params.argtypes = [_vp, _vp, ctypes.c_size_t]
_lib.fps_mlp_get_params.argtypes = [_vp, _vp, ctypes.c_size_t]
_lib.fps_mlp_predict.argtypes = [_vp, _vp, _i32, _vp, _vp]
_lib.fps_mlp_grad.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_float, _vp, _vp, _vp]
_lib.fps_mlp_train_step.argtypes = [_vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float, _vp, _vp]
_lib.fps_pack_query.argtypes = [ctypes.c_char_p, _vp]
_lib.fps_tune_class.argtypes = [_i32, _i32, _i32, ctypes.c_char_p]
_lib.fps_tune_cache_get.argtypes = [ctypes.c_char_p, ctypes.c_char_p, _i64, ctypes.c_char_p, ctypes.POINTER(_i32),
                                    ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)]
_lib.fps_tune_cache_put.argtypes = [ctypes.c_char_p, ctypes.c_char_p, _i64, ctypes.c_char_p, _i32, _i32,
                                    ctypes.c_double]
_lib.fps_pack_text.argtypes = [_vp, ctypes.c_size_t, ctypes.c_uint32, _vp, _vp, ctypes.c_size_t,
                               ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
for _f in ("fps_library_load", "fps_release", "fps_library_info_get", "fps_library_cid", "fps_search",
           "fps_search_packed", "fps_search_batch", "fps_sync", "fps_pack_query", "fps_pack_text", "fps_search_noalloc",
           "fps_mlp_create", "fps_mlp_release", "fps_mlp_set_params", "fps_mlp_get_params", "fps_mlp_predict",
           "fps_mlp_grad", "fps_mlp_train_step", "fps_merge_topk", "fps_batch_plan_create", "fps_batch_plan_run",
           "fps_batch_plan_release", "fps_search_shards", "fps_wide_load", "fps_wide_info", "fps_wide_search",
           "fps_wide_release", "fps_cluster_search"):
    getattr(_lib, _f).restype = _i32


def _check(st: int, where: str, line: int = 0):
    if st != FPS_OK:
        raise FpsError(st, where, line)


def library_path() -> str:
    return _SO


class Library:
    """A resident library handle (owns its device memory until fps_release)."""

    def __init__(self, handle: int):
        self.handle = handle

    @property
    def _h(self):
        if not self.handle:
            raise FpsError(FPS_ERR_INVALID_ARG, "released library")
        return self.handle

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        fps_release(self)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def _is_cuda(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def fps_library_load(*, path=None, text=None, packed=None, cids=None, device: int = 0, hbm_budget_bytes: int = 0,
                     flags: int = 0) -> Library:
    d = fps_load_desc()
    keep = []
    if path is not None:
        d.path = os.fsencode(path)
    if text is not None:
        buf = np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else \
            np.ascontiguousarray(text, dtype=np.uint8)
        keep.append(buf)
        d.text = buf.ctypes.data if buf.size else ctypes.addressof(ctypes.c_char(0))
        d.text_len = buf.size
    if packed is not None:
        p = np.ascontiguousarray(np.asarray(packed, dtype=np.uint64).reshape(-1, FPS_WORDS))
        keep.append(p)
        d.packed = p.ctypes.data if p.size else ctypes.addressof(ctypes.c_uint64(0))
        d.n_packed = p.shape[0]
        if cids is not None:
            c = np.ascontiguousarray(np.asarray(cids, dtype=np.int64))
            keep.append(c)
            d.cids = c.ctypes.data
    d.device, d.hbm_budget_bytes, d.flags = device, hbm_budget_bytes, flags
    err = ctypes.c_size_t(0)
    d.err_line = ctypes.pointer(err)
    h = _vp()
    st = _lib.fps_library_load(ctypes.byref(d), ctypes.byref(h))
    _check(st, "fps_library_load", err.value)
    return Library(h.value)


def fps_release(lib: Library):
    if lib is not None and lib.handle:
        _check(_lib.fps_release(lib.handle), "fps_release")
        lib.handle = None


def fps_library_info_get(lib: Library) -> dict:
    info = fps_library_info()
    _check(_lib.fps_library_info_get(lib._h, ctypes.byref(info)), "fps_library_info_get")
    return {"n_records": info.n_records, "n_tiles": info.n_tiles, "device_bytes": info.device_bytes,
            "device": info.device, "bucketed": bool(info.bucketed), "has_tc_operand": bool(info.has_tc_operand),
            "has_tc_fp4": bool(info.has_tc_fp4),
            "bucket_count": np.array(info.bucket_count[:], np.int64)}


def fps_tune_class(Q: int, k_max: int, learned: bool = False) -> str:
    """Autotuner size class of a batch (see include/fps.h)."""
    buf = ctypes.create_string_buffer(FPS_TUNE_CLASS_LEN)
    _check(_lib.fps_tune_class(int(Q), int(k_max), int(bool(learned)), buf), "fps_tune_class")
    return buf.value.decode()


def fps_tune_cache_get(path: str, device: str, n: int, cls: str):
    """(fps_path, tile_param, ms) of a cache entry, or None when the file or entry does not exist."""
    p, t, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    st = _lib.fps_tune_cache_get(os.fsencode(path), device.encode(), int(n), cls.encode(), ctypes.byref(p),
                                 ctypes.byref(t), ctypes.byref(ms))
    if st == FPS_ERR_IO:
        return None
    _check(st, "fps_tune_cache_get")
    return p.value, t.value, ms.value


def fps_tune_cache_put(path: str, device: str, n: int, cls: str, path_code: int, tile_param: int, ms: float):
    """Merge one autotuner choice into a cache file (created if missing)."""
    _check(_lib.fps_tune_cache_put(os.fsencode(path), device.encode(), int(n), cls.encode(), int(path_code),
                                   int(tile_param), float(ms)), "fps_tune_cache_put")


def fps_library_cid(lib: Library, index: int) -> int:
    c = _i64(0)
    _check(_lib.fps_library_cid(lib._h, int(index), ctypes.byref(c)), "fps_library_cid")
    return c.value


def fps_search(lib: Library, query166: str, k: int, stream=None):
    """The paper's single-molecule search: (index, distance, cid) NumPy arrays, ascending."""
    q = query166.encode() if isinstance(query166, str) else bytes(query166)
    if len(q) != FPS_BITS:
        raise FpsError(FPS_ERR_INVALID_ARG, "fps_search: query must have 166 characters")
    n = max(int(k), 1)
    idx, dist, cid = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int64)
    cnt = _i32(0)
    st = _lib.fps_search(lib._h, q, int(k), idx.ctypes.data, dist.ctypes.data, cid.ctypes.data,
                         ctypes.byref(cnt), _stream_ptr(stream))
    _check(st, "fps_search")
    c = cnt.value
    return idx[:c], dist[:c], cid[:c]


def _opts(path, flags, timeout_s, stats, tau_ptr=None):
    o = fps_search_opts()
    o.path, o.flags, o.timeout_s = int(path), int(flags), float(timeout_s)
    if stats is not None:
        o.stats = ctypes.pointer(stats)
    if tau_ptr:
        o.tau = tau_ptr
    return o


def fps_search_packed(lib: Library, query, k: int, *, out_index=None, out_dist=None, out_count=None,
                      path: int = FPS_PATH_POPC, timeout_s: float = 0.0, stream=None):
    """Single packed query (3 uint64 words).

    Host form: ``query`` is a NumPy array; returns (index, distance) NumPy arrays.
    Device form: ``query`` is a CUDA tensor; outputs are CUDA int32 tensors
    (allocated if not given) and the call is asynchronous on ``stream``;
    returns (out_index, out_dist, out_count).
    """
    if _is_cuda(query):
        import torch

        dev = query.device
        if out_index is None:
            out_index = torch.empty(max(int(k), 1), dtype=torch.int32, device=dev)
        if out_dist is None:
            out_dist = torch.empty(max(int(k), 1), dtype=torch.int32, device=dev)
        if out_count is None:
            out_count = torch.empty(1, dtype=torch.int32, device=dev)
        o = _opts(path, FPS_SEARCH_DEVICE_IO, timeout_s, None)
        st = _lib.fps_search_packed(lib._h, query.data_ptr(), int(k), out_index.data_ptr(), out_dist.data_ptr(),
                                    out_count.data_ptr(), ctypes.byref(o), _stream_ptr(stream))
        _check(st, "fps_search_packed")
        return out_index, out_dist, out_count
    q = np.ascontiguousarray(np.asarray(query, dtype=np.uint64).reshape(FPS_WORDS))
    n = max(int(k), 1)
    idx, dist, cnt = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(1, np.int32)
    stats = fps_search_stats()
    o = _opts(path, 0, timeout_s, stats)
    st = _lib.fps_search_packed(lib._h, q.ctypes.data, int(k), idx.ctypes.data, dist.ctypes.data, cnt.ctypes.data,
                                ctypes.byref(o), _stream_ptr(stream))
    _check(st, "fps_search_packed")
    return idx[: cnt[0]], dist[: cnt[0]]


def batch_offsets(k) -> np.ndarray:
    k = np.asarray(k, dtype=np.int64).reshape(-1)
    off = np.zeros(k.size + 1, np.int64)
    off[1:] = np.cumsum(np.maximum(k, 0))
    return off


def fps_search_batch(lib: Library, queries, k, *, path: int = FPS_PATH_AUTO, out_index=None, out_dist=None,
                     out_count=None, offsets=None, tau=None, timeout_s: float = 0.0, stream=None, stats=None,
                     flat: bool = False):
    """Many packed queries (Q x 3 uint64) with per-query k (host array or scalar).

    Host form (NumPy queries): returns a list of (index, distance) per query, or with flat=True
    the arrays (index, distance, count, offsets) without per-query copies.
    Device form (CUDA tensor queries): outputs are CUDA int32 tensors laid out
    by ``offsets`` (prefix sums of k); asynchronous; returns
    (out_index, out_dist, out_count, offsets).
    """
    Q = int(queries.shape[0]) if hasattr(queries, "shape") else len(queries)
    kk = np.asarray(k, dtype=np.int32).reshape(-1)
    if kk.size == 1 and Q != 1:
        kk = np.full(Q, kk[0], np.int32)
    kk = np.ascontiguousarray(kk)
    off = batch_offsets(kk) if offsets is None else np.ascontiguousarray(np.asarray(offsets, np.int64))
    total = max(int(off[-1]), 1)
    st_obj = stats if stats is not None else fps_search_stats()
    if _is_cuda(queries):
        import torch

        dev = queries.device
        if out_index is None:
            out_index = torch.empty(total, dtype=torch.int32, device=dev)
        if out_dist is None:
            out_dist = torch.empty(total, dtype=torch.int32, device=dev)
        if out_count is None:
            out_count = torch.empty(max(Q, 1), dtype=torch.int32, device=dev)
        o = _opts(path, FPS_SEARCH_DEVICE_IO, timeout_s, st_obj, tau.data_ptr() if tau is not None else None)
        st = _lib.fps_search_batch(lib._h, queries.data_ptr(), Q, kk.ctypes.data, off.ctypes.data,
                                   out_index.data_ptr(), out_dist.data_ptr(), out_count.data_ptr(), ctypes.byref(o),
                                   _stream_ptr(stream))
        _check(st, "fps_search_batch")
        return out_index, out_dist, out_count, off
    q = np.ascontiguousarray(np.asarray(queries, dtype=np.uint64).reshape(-1, FPS_WORDS))
    idx, dist, cnt = np.zeros(total, np.int32), np.zeros(total, np.int32), np.zeros(max(Q, 1), np.int32)
    tau_arr = None
    if tau is not None:
        tau_arr = np.ascontiguousarray(np.asarray(tau, np.float32))
    o = _opts(path, 0, timeout_s, st_obj, tau_arr.ctypes.data if tau_arr is not None else None)
    st = _lib.fps_search_batch(lib._h, q.ctypes.data, Q, kk.ctypes.data, off.ctypes.data, idx.ctypes.data,
                               dist.ctypes.data, cnt.ctypes.data, ctypes.byref(o), _stream_ptr(stream))
    _check(st, "fps_search_batch")
    if flat:
        return idx, dist, cnt, off
    return [(idx[off[i]: off[i] + cnt[i]].copy(), dist[off[i]: off[i] + cnt[i]].copy()) for i in range(Q)]


def fps_search_noalloc(lib: Library, query, k: int, out_index, out_dist, out_count, stream=None):
    """Single packed query into caller-owned CUDA tensors, with no device allocation by the library.

    For callers that cannot allocate device memory while searching (see
    include/fps.h).  ``query`` (3 x 64-bit), ``out_index``/``out_dist`` (>= k int32)
    and ``out_count`` (1 int32) are CUDA tensors; asynchronous on ``stream``.
    Calls on one device share the library's fixed scratch array, so they must not
    overlap on the GPU.  ``out_count == -1`` after the stream completes means the
    search failed on the device.
    """
    st = _lib.fps_search_noalloc(lib._h, query.data_ptr(), int(k), out_index.data_ptr(), out_dist.data_ptr(),
                                 out_count.data_ptr(), _stream_ptr(stream))
    _check(st, "fps_search_noalloc")
    return out_index, out_dist, out_count


FPS_SHARDS_MAX = 32


def shard_progress(n: int):
    """Pinned host int64[n] (a CPU torch tensor) for fps_search_shards to report per-shard progress into."""
    import torch

    return torch.zeros(n, dtype=torch.int64, pin_memory=True)


def fps_search_shards(libs, queries, k, *, index_base=None, path: int = FPS_PATH_AUTO, out_index=None, out_dist=None,
                      out_count=None, offsets=None, progress=None, timeout_s: float = 0.0, stream=None, stats=None):
    """Several resident libraries searched as one, results merged with global indices.

    libs: Library handles; library s holds global indices index_base[s] .. (default: the prefix sums of
    their sizes).  Forms and outputs as in fps_search_batch.  progress: a tensor from shard_progress();
    entry s becomes Q once shard s's results are complete.
    """
    n = len(libs)
    harr = (ctypes.c_void_p * max(n, 1))(*[lb._h for lb in libs])
    base = None if index_base is None else np.ascontiguousarray(np.asarray(index_base, np.int64))
    Q = int(queries.shape[0]) if hasattr(queries, "shape") else len(queries)
    kk = np.asarray(k, dtype=np.int32).reshape(-1)
    if kk.size == 1 and Q != 1:
        kk = np.full(Q, kk[0], np.int32)
    kk = np.ascontiguousarray(kk)
    off = batch_offsets(kk) if offsets is None else np.ascontiguousarray(np.asarray(offsets, np.int64))
    total = max(int(off[-1]), 1)
    st_obj = stats if stats is not None else fps_search_stats()
    prog = progress.data_ptr() if progress is not None else None
    bptr = base.ctypes.data if base is not None else None
    if _is_cuda(queries):
        import torch

        dev = queries.device
        if out_index is None:
            out_index = torch.empty(total, dtype=torch.int32, device=dev)
        if out_dist is None:
            out_dist = torch.empty(total, dtype=torch.int32, device=dev)
        if out_count is None:
            out_count = torch.empty(max(Q, 1), dtype=torch.int32, device=dev)
        o = _opts(path, FPS_SEARCH_DEVICE_IO, timeout_s, st_obj)
        _check(_lib.fps_search_shards(harr, n, bptr, queries.data_ptr(), Q, kk.ctypes.data, off.ctypes.data,
                                      out_index.data_ptr(), out_dist.data_ptr(), out_count.data_ptr(), ctypes.byref(o),
                                      prog, _stream_ptr(stream)), "fps_search_shards")
        return out_index, out_dist, out_count, off
    q = np.ascontiguousarray(np.asarray(queries, dtype=np.uint64).reshape(-1, FPS_WORDS))
    idx, dist, cnt = np.zeros(total, np.int32), np.zeros(total, np.int32), np.zeros(max(Q, 1), np.int32)
    o = _opts(path, 0, timeout_s, st_obj)
    _check(_lib.fps_search_shards(harr, n, bptr, q.ctypes.data, Q, kk.ctypes.data, off.ctypes.data, idx.ctypes.data,
                                  dist.ctypes.data, cnt.ctypes.data, ctypes.byref(o), prog, _stream_ptr(stream)),
           "fps_search_shards")
    return [(idx[off[i]: off[i] + cnt[i]].copy(), dist[off[i]: off[i] + cnt[i]].copy()) for i in range(Q)]


def fps_merge_topk(parts, k: int):
    """Merge per-shard (index, distance) lists (each ascending, global indices) into the combined top-k."""
    idx = np.ascontiguousarray(np.concatenate([np.asarray(a, np.int32) for a, _ in parts] or [np.zeros(0, np.int32)]))
    dist = np.ascontiguousarray(np.concatenate([np.asarray(b, np.int32) for _, b in parts] or [np.zeros(0, np.int32)]))
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([len(a) for a, _ in parts])
    oi, od = np.zeros(max(k, 1), np.int32), np.zeros(max(k, 1), np.int32)
    n = _i32(0)
    _check(_lib.fps_merge_topk(idx.ctypes.data if idx.size else None, dist.ctypes.data if dist.size else None,
                               off.ctypes.data, len(parts), int(k), oi.ctypes.data, od.ctypes.data, ctypes.byref(n)),
           "fps_merge_topk")
    return oi[: n.value], od[: n.value]


def fps_sync(lib: Library, stream=None):
    _check(_lib.fps_sync(lib._h, _stream_ptr(stream)), "fps_sync")


def fps_pack_query(query166: str) -> np.ndarray:
    out = np.zeros(FPS_WORDS, np.uint64)
    q = query166.encode() if isinstance(query166, str) else bytes(query166)
    if len(q) != FPS_BITS:
        raise FpsError(FPS_ERR_INVALID_ARG, "fps_pack_query: query must have 166 characters")
    _check(_lib.fps_pack_query(q, out.ctypes.data), "fps_pack_query")
    return out


def fps_pack_text(text, flags: int = 0):
    """Host-only parse of library text: (packed uint64[N, 3], cids int64[N])."""
    buf = np.frombuffer(bytes(text), dtype=np.uint8)
    ptr = buf.ctypes.data if buf.size else None
    n = ctypes.c_size_t(0)
    err = ctypes.c_size_t(0)
    st = _lib.fps_pack_text(ptr, buf.size, flags, None, None, 0, ctypes.byref(n), ctypes.byref(err))
    _check(st, "fps_pack_text", err.value)
    packed = np.zeros((max(n.value, 1), FPS_WORDS), np.uint64)
    cids = np.zeros(max(n.value, 1), np.int64)
    st = _lib.fps_pack_text(ptr, buf.size, flags, packed.ctypes.data, cids.ctypes.data, n.value, ctypes.byref(n),
                            ctypes.byref(err))
    _check(st, "fps_pack_text", err.value)
    return packed[: n.value], cids[: n.value]


# ------------------------------------------------------------ learned threshold MLP
class Mlp:
    """Threshold-predicting MLP handle (device weights)."""

    def __init__(self, handle: int):
        self.handle = handle

    @property
    def _h(self):
        if not self.handle:
            raise FpsError(FPS_ERR_INVALID_ARG, "released model")
        return self.handle


def fps_mlp_param_count() -> int:
    return int(_lib.fps_mlp_param_count())


def fps_mlp_create(device: int = 0) -> Mlp:
    h = _vp()
    _check(_lib.fps_mlp_create(device, ctypes.byref(h)), "fps_mlp_create")
    return Mlp(h.value)


def fps_mlp_release(m: Mlp):
    if m is not None and m.handle:
        _check(_lib.fps_mlp_release(m.handle), "fps_mlp_release")
        m.handle = None


def fps_mlp_set_params(m: Mlp, params) -> None:
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    _check(_lib.fps_mlp_set_params(m._h, p.ctypes.data, p.size), "fps_mlp_set_params")


def fps_mlp_get_params(m: Mlp) -> np.ndarray:
    p = np.zeros(fps_mlp_param_count(), np.float32)
    _check(_lib.fps_mlp_get_params(m._h, p.ctypes.data, p.size), "fps_mlp_get_params")
    return p


def fps_mlp_predict(m: Mlp, queries, out=None, stream=None):
    """queries: CUDA int64/uint64 tensor [Q, 3]; returns a CUDA float32 tensor [Q] (asynchronous)."""
    import torch

    Q = int(queries.shape[0])
    if out is None:
        out = torch.empty(max(Q, 1), dtype=torch.float32, device=queries.device)
    _check(_lib.fps_mlp_predict(m._h, queries.data_ptr(), Q, out.data_ptr(), _stream_ptr(stream)), "fps_mlp_predict")
    return out


def fps_mlp_grad(m: Mlp, queries, targets, quantile: float, stream=None):
    """(mean loss, flat FP32 gradient) for device queries [B, 3] and targets [B]."""
    g = np.zeros(fps_mlp_param_count(), np.float32)
    loss = np.zeros(1, np.float32)
    _check(_lib.fps_mlp_grad(m._h, queries.data_ptr(), targets.data_ptr(), int(queries.shape[0]), float(quantile),
                             g.ctypes.data, loss.ctypes.data, _stream_ptr(stream)), "fps_mlp_grad")
    return float(loss[0]), g


def fps_mlp_train_step(m: Mlp, queries, targets, quantile: float, lr: float, want_loss: bool = False, stream=None):
    loss = np.zeros(1, np.float32)
    _check(_lib.fps_mlp_train_step(m._h, queries.data_ptr(), targets.data_ptr(), int(queries.shape[0]),
                                   float(quantile), float(lr), loss.ctypes.data if want_loss else None,
                                   _stream_ptr(stream)), "fps_mlp_train_step")
    return float(loss[0]) if want_loss else None


# ------------------------------------------------------------ graph-captured batch plan
class BatchPlan:
    def __init__(self, handle, k):
        self.handle = handle
        self.k = np.ascontiguousarray(np.asarray(k, np.int32))
        self.off = batch_offsets(self.k)


def fps_batch_plan_create(lib: Library, k, path: int = FPS_PATH_AUTO, learned: bool = False) -> BatchPlan:
    kk = np.ascontiguousarray(np.asarray(k, np.int32).reshape(-1))
    h = _vp()
    _check(_lib.fps_batch_plan_create(lib._h, kk.size, kk.ctypes.data, int(path), int(learned), ctypes.byref(h)),
           "fps_batch_plan_create")
    return BatchPlan(h.value, kk)


def fps_batch_plan_run(plan: BatchPlan, queries, tau=None, stats=None, stream=None, flat: bool = False):
    """Run a captured batch on host queries [Q, 3]; returns a list of (index, distance) per query, or with
    flat=True the arrays (index, distance, count, offsets): query i's results are
    index[offsets[i]: offsets[i] + count[i]] (no per-query copies)."""
    q = np.ascontiguousarray(np.asarray(queries, dtype=np.uint64).reshape(-1, FPS_WORDS))
    Q = plan.k.size
    total = max(int(plan.off[-1]), 1)
    idx, dist, cnt = np.zeros(total, np.int32), np.zeros(total, np.int32), np.zeros(Q, np.int32)
    t = np.ascontiguousarray(np.asarray(tau, np.float32)) if tau is not None else None
    st_obj = stats if stats is not None else fps_search_stats()
    _check(_lib.fps_batch_plan_run(plan.handle, q.ctypes.data, t.ctypes.data if t is not None else None,
                                   idx.ctypes.data, dist.ctypes.data, cnt.ctypes.data, ctypes.byref(st_obj),
                                   _stream_ptr(stream)), "fps_batch_plan_run")
    off = plan.off
    if flat:
        return idx, dist, cnt, off
    return [(idx[off[i]: off[i] + cnt[i]].copy(), dist[off[i]: off[i] + cnt[i]].copy()) for i in range(Q)]


def fps_batch_plan_release(plan: BatchPlan):
    if plan is not None and plan.handle:
        _check(_lib.fps_batch_plan_release(plan.handle), "fps_batch_plan_release")
        plan.handle = None


# ------------------------------------------------------------------ wide
FPS_WIDE_MAX_BITS, FPS_METRIC_MANHATTAN, FPS_METRIC_TANIMOTO = 2048, 0, 1


class WideLibrary(Library):
    """A resident library of n-bit fingerprints (owns its device memory until fps_wide_release)."""

    def __init__(self, handle: int, n_bits: int):
        super().__init__(handle)
        self.n_bits = n_bits
        self.words = (n_bits + 63) // 64

    def __exit__(self, *exc):
        fps_wide_release(self)


def fps_wide_load(*, text=None, packed=None, n_bits: int, device: int = 0, hbm_budget_bytes: int = 0) -> WideLibrary:
    """Load text (lines of n_bits '0'/'1' characters) or packed words (uint64 [N, W]) into device memory."""
    h = _vp()
    err = ctypes.c_size_t(0)
    if text is not None:
        buf = text if isinstance(text, (bytes, bytearray)) else bytes(text)
        st = _lib.fps_wide_load(buf, len(buf), None, 0, int(n_bits), int(device), int(hbm_budget_bytes),
                                ctypes.byref(h), ctypes.byref(err))
    else:
        # the library checks n_bits; a shape for the reshape even when it is out of range
        pk = np.ascontiguousarray(np.asarray(packed, np.uint64).reshape(-1, max((int(n_bits) + 63) // 64, 1)))
        st = _lib.fps_wide_load(None, 0, pk.ctypes.data, pk.shape[0], int(n_bits), int(device), int(hbm_budget_bytes),
                                ctypes.byref(h), ctypes.byref(err))
    _check(st, "fps_wide_load", err.value)
    return WideLibrary(h.value, int(n_bits))


def fps_wide_info(lib: WideLibrary) -> dict:
    n, b, db = _i64(0), _i32(0), ctypes.c_size_t(0)
    _check(_lib.fps_wide_info(lib._h, ctypes.byref(n), ctypes.byref(b), ctypes.byref(db)), "fps_wide_info")
    return {"n_records": n.value, "n_bits": b.value, "device_bytes": db.value}


def fps_wide_search(lib: WideLibrary, query, k: int, metric: int = FPS_METRIC_MANHATTAN, *, out_index=None,
                    out_num=None, out_den=None, out_count=None, stream=None):
    """Host form (NumPy query of W words): returns (index, num, den) with the measure num / den
    (Manhattan d / 1, Tanimoto c / u).  Device form (CUDA tensor query): asynchronous on stream; returns
    (out_index, out_num, out_den, out_count) CUDA int32 tensors."""
    if _is_cuda(query):
        import torch

        dev = query.device
        m = max(int(k), 1)
        out_index = out_index if out_index is not None else torch.empty(m, dtype=torch.int32, device=dev)
        out_num = out_num if out_num is not None else torch.empty(m, dtype=torch.int32, device=dev)
        out_den = out_den if out_den is not None else torch.empty(m, dtype=torch.int32, device=dev)
        out_count = out_count if out_count is not None else torch.empty(1, dtype=torch.int32, device=dev)
        _check(_lib.fps_wide_search(lib._h, query.data_ptr(), int(k), int(metric), out_index.data_ptr(),
                                    out_num.data_ptr(), out_den.data_ptr(), out_count.data_ptr(), FPS_SEARCH_DEVICE_IO,
                                    _stream_ptr(stream)), "fps_wide_search")
        return out_index, out_num, out_den, out_count
    q = np.ascontiguousarray(np.asarray(query, np.uint64).reshape(lib.words))
    m = max(int(k), 1)
    idx, num, den, cnt = np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(1, np.int32)
    _check(_lib.fps_wide_search(lib._h, q.ctypes.data, int(k), int(metric), idx.ctypes.data, num.ctypes.data,
                                den.ctypes.data, cnt.ctypes.data, 0, _stream_ptr(stream)), "fps_wide_search")
    c = int(cnt[0])
    return idx[:c], num[:c], den[:c]


def fps_wide_release(lib: WideLibrary):
    if lib is not None and lib.handle:
        _check(_lib.fps_wide_release(lib.handle), "fps_wide_release")
        lib.handle = None


# ------------------------------------------------------------------ batch clustering
FPS_CLUSTER_MAX_Q, FPS_CLUSTER_MAX_C = 4096, 16


def fps_cluster_search(lib: Library, queries, k: int = 30, c_min: int = 2, c_max: int = 8, stream=None) -> dict:
    """Batch clustering search (host arrays): cluster the packed queries [Q, 3] by k-medoids with the count
    chosen by the silhouette, then the k nearest library records of every cluster's medoid.  Returns
    {"c", "labels" [Q], "medoids" [c], "scores" {c: sum floor(s * 2^32)}, "results" [(index, distance)] * c}."""
    q = np.ascontiguousarray(np.asarray(queries, np.uint64).reshape(-1, FPS_WORDS))
    Q = q.shape[0]
    n_c = max(int(c_max) - int(c_min) + 1, 1)
    c = _i32(0)
    labels = np.zeros(max(Q, 1), np.int32)
    medoids = np.zeros(FPS_CLUSTER_MAX_C, np.int32)
    scores = np.zeros(n_c, np.int64)
    m = max(int(k), 1)
    idx = np.zeros(FPS_CLUSTER_MAX_C * m, np.int32)
    dist = np.zeros(FPS_CLUSTER_MAX_C * m, np.int32)
    cnt = np.zeros(FPS_CLUSTER_MAX_C, np.int32)
    _check(_lib.fps_cluster_search(lib._h, q.ctypes.data, Q, int(c_min), int(c_max), int(k), ctypes.byref(c),
                                   labels.ctypes.data, medoids.ctypes.data, scores.ctypes.data, idx.ctypes.data,
                                   dist.ctypes.data, cnt.ctypes.data, _stream_ptr(stream)), "fps_cluster_search")
    cc = c.value
    kk = int(k)
    return {"c": cc, "labels": labels[:Q].copy(), "medoids": medoids[:cc].copy(),
            "scores": {int(c_min) + i: int(v) for i, v in enumerate(scores) if v != np.iinfo(np.int64).min},
            "results": [(idx[t * kk: t * kk + cnt[t]].copy(), dist[t * kk: t * kk + cnt[t]].copy()) for t in range(cc)]}
