"""Serving loop: queued single-molecule requests against several resident libraries.

The paper decouples its web tier from the compute back end with a queue
(Sec. 3.1, "interact with each other in a queuing way") and runs each search
to completion (Sec. 4.4).  Here the back end is one process holding several
libraries in GPU memory; requests arrive over time, wait in one queue per
library, and are served in dynamic batches (up to max_batch requests of one
library per call, oldest library first) through fps_search_batch.  A request
carries one query (shape [3]) or several (shape [m, 3], all with the request's
k); a batch takes whole requests while their queries fit in max_batch.  The
plain baseline serves the same arrivals one request at a time with
fps_search_packed.  Latency = completion - arrival, on the host clock.

Only host-side scheduling lives here; every search step runs in the library's
CUDA kernels.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import FPS_PATH_AUTO, FPS_PATH_POPC, FPS_PATH_POPC_BATCH, fps_search_batch, fps_search_packed


class Request:
    """result: (index, distance) for a one-query request, a list of them for a [m, 3] request."""
    __slots__ = ("arrival", "lib", "query", "k", "done", "result")

    def __init__(self, arrival, lib, query, k):
        self.arrival, self.lib, self.query, self.k = arrival, lib, query, k
        self.done = None
        self.result = None

    @property
    def nq(self) -> int:
        return 1 if np.ndim(self.query) == 1 else int(np.shape(self.query)[0])


def choose_path(q: int, has_tc: bool) -> int:
    """Path for a batch of q queries: one query -> single-query scan; small batches -> popcount batch;
    64 or more -> tensor cores when the library holds the FP8 operand."""
    if q == 1:
        return FPS_PATH_POPC
    if q >= 64 and has_tc:
        return FPS_PATH_AUTO
    return FPS_PATH_POPC_BATCH


class Server:
    """libraries: name -> Library.  batch_fn(name, queries [B, 3], ks [B]) and one_fn(name, query, k) default
    to the library's batched and single-query searches; tests may pass stand-ins."""

    def __init__(self, libraries: dict, has_tc: dict | None = None, max_batch: int = 512, batch_fn=None,
                 one_fn=None):
        self.libraries = libraries
        self.has_tc = has_tc or {name: False for name in libraries}
        self.max_batch = max_batch
        self.batch_fn = batch_fn or (lambda name, qs, ks: fps_search_batch(
            self.libraries[name], qs, ks, path=choose_path(len(ks), self.has_tc[name])))
        self.one_fn = one_fn or (lambda name, q, k: fps_search_packed(self.libraries[name], q, k))
        self.batch_sizes = []

    def _serve_batch(self, name, reqs):
        qs = np.concatenate([np.reshape(r.query, (-1, 3)) for r in reqs])
        ks = np.concatenate([np.full(r.nq, r.k, np.int32) for r in reqs])
        self.batch_sizes.append(len(ks))
        res = self.batch_fn(name, qs, ks)
        now = time.perf_counter()
        pos = 0
        for r in reqs:
            r.done = now
            r.result = res[pos] if np.ndim(r.query) == 1 else list(res[pos: pos + r.nq])
            pos += r.nq

    def run(self, requests, batched: bool = True, keep_results: bool = True):
        """Replay requests (sorted by arrival, seconds from start) in real time; returns them completed."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        queues = {name: collections.deque() for name in self.libraries}
        t0 = time.perf_counter()
        for r in reqs:
            r.arrival += t0
        i, n, served = 0, len(reqs), 0
        while served < n:
            now = time.perf_counter()
            while i < n and reqs[i].arrival <= now:
                queues[reqs[i].lib].append(reqs[i])
                i += 1
            live = [nm for nm, q in queues.items() if q]
            if not live:
                if i < n:
                    wait = reqs[i].arrival - time.perf_counter()
                    if wait > 2e-4:
                        time.sleep(wait - 1e-4)
                continue
            name = min(live, key=lambda nm: queues[nm][0].arrival)      # oldest waiting request first
            q = queues[name]
            if batched:
                batch, total = [q.popleft()], 0
                total = batch[0].nq
                while q and total + q[0].nq <= self.max_batch:
                    total += q[0].nq
                    batch.append(q.popleft())
                self._serve_batch(name, batch)
                served += len(batch)
            else:
                r = q.popleft()
                r.result = self.one_fn(name, r.query, r.k)
                r.done = time.perf_counter()
                served += 1
        for r in reqs:
            r.arrival -= t0
            r.done -= t0
            if not keep_results:
                r.result = None
        return reqs


def latency_stats(reqs):
    lat = np.array([r.done - r.arrival for r in reqs])
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    nq = sum(r.nq for r in reqs)
    return {"requests": len(reqs), "queries": nq, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "throughput_rps": len(reqs) / span if span > 0 else float("nan"),
            "throughput_qps": nq / span if span > 0 else float("nan"), "span_s": span}


def poisson_arrivals(n: int, rate: float, seed: int):
    """n arrival times (seconds) of a Poisson process with the given rate (exponential gaps, seeded)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))
