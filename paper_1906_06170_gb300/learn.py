"""Learned per-query threshold: label generation, training, calibration, checkpoints.

Host-side orchestration only; every numeric step runs in the library's CUDA
kernels (exact labels from the batched search, forward/backward/Adam of the
MLP from fps_mlp_*).  The model predicts a query's k-th-nearest distance; the
batched search with FPS_PATH_LEARNED starts each query from that bound and
re-runs any query whose bound turned out too low, so results stay exact.
"""
from __future__ import annotations

import json
import struct
import zlib

import numpy as np

from . import (FPS_PATH_AUTO, FPS_PATH_LEARNED, batch_offsets, fps_mlp_create, fps_mlp_get_params,
               fps_mlp_param_count, fps_mlp_predict, fps_mlp_set_params, fps_mlp_train_step, fps_search_batch,
               fps_search_stats)

MAGIC = b"FPSMLP01"


def exact_kth(lib, queries, k: int, path: int = FPS_PATH_AUTO, chunk: int = 4096):
    """Exact k-th smallest distance of every query (CUDA int64 tensor [Q, 3]) -> CUDA float32 [Q]."""
    import torch

    Q = int(queries.shape[0])
    out = torch.empty(Q, dtype=torch.float32, device=queries.device)
    for lo in range(0, Q, chunk):
        q = queries[lo: lo + chunk]
        ks = np.full(q.shape[0], k, np.int32)
        oi, od, oc, off = fps_search_batch(lib, q, ks, path=path)
        out[lo: lo + q.shape[0]] = od.view(-1, k)[:, k - 1].float()
    return out


def init_params(seed: int = 0, bias_out: float = 20.0) -> np.ndarray:
    """He-normal weights, zero hidden biases, output bias near a typical distance."""
    rng = np.random.default_rng(seed)
    h, n_in = 256, 167
    parts = [rng.standard_normal((h, n_in)) * np.sqrt(2.0 / n_in), np.zeros(h),
             rng.standard_normal((h, h)) * np.sqrt(2.0 / h), np.zeros(h),
             rng.standard_normal(h) * np.sqrt(1.0 / h), np.array([bias_out])]
    flat = np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)
    assert flat.size == fps_mlp_param_count()
    return flat


def train(model, queries, targets, epochs: int = 8, batch: int = 4096, lr: float = 2e-3, quantile: float = 0.9,
          seed: int = 0, log_every: int = 0):
    """Minibatch Adam on (queries [N, 3] CUDA int64, targets [N] CUDA float32); returns per-epoch mean losses."""
    import torch

    n = int(queries.shape[0])
    g = torch.Generator(device="cpu").manual_seed(seed)
    history = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(queries.device)
        losses = []
        for i, lo in enumerate(range(0, n - batch + 1, batch)):
            idx = perm[lo: lo + batch]
            qb = queries.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
            want = (i % 50 == 0)
            loss = fps_mlp_train_step(model, qb, tb, quantile, lr, want_loss=want)
            if want:
                losses.append(loss)
        history.append(float(np.mean(losses)) if losses else float("nan"))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: pinball loss {history[-1]:.4f}", flush=True)
    return history


def offset_for(pred, targets, max_fallback: float = 0.002) -> float:
    """Smallest integer offset delta with P(ceil(pred + delta) < target) <= max_fallback."""
    pred = np.asarray(pred, np.float64)
    t = np.asarray(targets, np.float64)
    for delta in range(-8, 40):
        if np.mean(np.ceil(pred + delta) < t) <= max_fallback:
            return float(delta)
    return 40.0


def calibrate_offset(model, queries, targets, max_fallback: float = 0.002) -> float:
    """offset_for() of the model's predictions on held-out queries (CUDA tensors)."""
    pred = fps_mlp_predict(model, queries).float().cpu().numpy()[: int(queries.shape[0])]
    return offset_for(pred, targets.float().cpu().numpy(), max_fallback)


def query_popcounts(queries) -> np.ndarray:
    """popc of packed queries (host uint64 [Q, 3], or a CUDA int64 tensor)."""
    if hasattr(queries, "cpu"):
        queries = queries.cpu().numpy()
    q = np.ascontiguousarray(np.asarray(queries).view(np.uint64).reshape(-1, 3))
    return np.unpackbits(q.view(np.uint8), axis=1, bitorder="little")[:, :166].sum(1).astype(np.int64)


def popc_quantile_table(queries, targets, quantile: float = 0.9) -> np.ndarray:
    """Non-learned predictor of the k-th distance: for each query popcount p (0..166), the given quantile
    of the training targets whose query has popcount p; popcounts with no training query take the
    value of the nearest popcount that has one."""
    pc = query_popcounts(queries)
    t = targets.float().cpu().numpy() if hasattr(targets, "cpu") else np.asarray(targets, np.float64)
    table = np.full(167, np.nan)
    for p in np.unique(pc):
        table[p] = np.quantile(t[pc == p], quantile)
    have = np.flatnonzero(~np.isnan(table))
    if have.size == 0:
        raise ValueError("no training targets")
    for p in np.flatnonzero(np.isnan(table)):
        table[p] = table[have[np.argmin(np.abs(have - p))]]
    return table.astype(np.float32)


def table_tau(table, queries, offset: float = 0.0) -> np.ndarray:
    """Bounds (float32 [Q]) from a popcount table, including an offset."""
    return (np.asarray(table, np.float32)[query_popcounts(queries)] + np.float32(offset)).astype(np.float32)


def predict_tau(model, queries, offset: float = 0.0):
    """Predicted bounds (CUDA float32 [Q]) including the calibration offset."""
    tau = fps_mlp_predict(model, queries)
    return tau[: int(queries.shape[0])] + offset


def learned_search(lib, model, queries, ks, offset: float = 0.0, stats=None, stream=None):
    """Batched exact search starting from the model's predicted bounds (device inputs and outputs)."""
    tau = predict_tau(model, queries, offset).contiguous()
    st = stats if stats is not None else fps_search_stats()
    res = fps_search_batch(lib, queries, ks, path=FPS_PATH_LEARNED, tau=tau, stats=st, stream=stream)
    return res, st


def save(model, path: str, meta: dict) -> None:
    """Checkpoint: magic, meta (JSON), FP32 parameters, CRC32 of everything before it."""
    params = fps_mlp_get_params(model)
    mj = json.dumps(meta, sort_keys=True).encode()
    body = MAGIC + struct.pack("<QI", params.size, len(mj)) + mj + params.astype("<f4").tobytes()
    with open(path, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))


def load(path: str, device: int = 0):
    """(model, meta) from a checkpoint written by save(); raises ValueError on a bad file."""
    data = open(path, "rb").read()
    if len(data) < 24 or data[:8] != MAGIC:
        raise ValueError("not an MLP checkpoint")
    body, crc = data[:-4], struct.unpack("<I", data[-4:])[0]
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError("checkpoint checksum mismatch")
    n, mlen = struct.unpack("<QI", body[8:20])
    meta = json.loads(body[20: 20 + mlen].decode())
    params = np.frombuffer(body[20 + mlen:], dtype="<f4")
    if params.size != n or n != fps_mlp_param_count():
        raise ValueError("checkpoint parameter count mismatch")
    model = fps_mlp_create(device)
    fps_mlp_set_params(model, params)
    return model, meta


__all__ = ["exact_kth", "init_params", "train", "offset_for", "calibrate_offset", "predict_tau", "learned_search",
           "query_popcounts", "popc_quantile_table", "table_tau", "save", "load", "batch_offsets"]
