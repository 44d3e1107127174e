"""Continuous-batching triangle-count service on one GPU.

A request is one graph (an edge list on the host, its vertex count and a root
rule).

- The **admission** thread takes every request that has arrived, in arrival order and up to
  ``max_batch``, while the requests' HBM footprints fit the budget next to everything already
  resident. It builds them on the device as one batch on its own stream: a single
  host-to-device copy of their edge lists, one radix sort, one concatenated CSR
  (``tc_batch_create_from_edges``). The batch is queued as ready.
- The **counting** thread counts ready batches one after another: one multi-source BFS and one
  pass of each count kernel per batch. It then answers each request and frees the batch. The memory
  returns to the budget for the next admissions.

While a batch is on the device, newly arrived graphs are being admitted and built for the next one.
Building and counting overlap on the device: the batch's memory, sort buffers included, comes
stream-ordered from the library's pool and goes back without a device-wide synchronisation, and
the edge lists are staged in page-locked host memory, so neither thread's copies, allocations or
frees wait for the other's kernels. The server records every build and count interval;
``overlap_stats`` reports how much of the build time ran while a count was in progress. A request
never waits for a fixed batch size.

Latency is measured from arrival to the moment the count is on the host; p50 / p99 come from the
completed requests.
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

import paper_2403_02997_gb300 as tc


def footprint_bytes(n: int, draws: int) -> int:
    """Device bytes one request may hold.

    This counts the graph handle (CSR, its row array, and the per-count state, with m <= draws
    undirected edges), its share of the batch union (a second copy of the same), and the
    transient sort buffers of the build (two arrays of 2·draws 8-byte keys plus the staged edge
    list).
    """
    per_graph = 8 * (n + 1) + 4 * (2 * draws + 8) + 68 * n + 44 * draws
    transient = 32 * draws + 8 * draws
    return 2 * per_graph + transient + (1 << 16)


@dataclass
class Request:
    rid: int
    src: np.ndarray
    dst: np.ndarray
    n: int
    root: Optional[int] = None          # None: the smallest id of largest degree
    arrival: float = 0.0                # time.perf_counter() at arrival
    done: float = 0.0
    count: Optional[int] = None
    error: Optional[str] = None
    bytes: int = 0
    event: threading.Event = field(default_factory=threading.Event)

    def latency(self) -> float:
        return self.done - self.arrival


class GpuBackend:
    """Builds an admitted group as one device batch and counts it (the library's batch calls).

    Builds run on one stream and counts on another, so a group builds while the previous one
    counts.
    """

    def __init__(self, params=None):
        import torch
        self.params = dict(params or {})
        self.build_stream = torch.cuda.Stream()
        self.count_stream = torch.cuda.Stream()
        self.staging = tc.PinnedStaging()   # used by the admission thread only

    def build(self, group):
        """One batch straight from the group's edge lists; returns (batch, roots)."""
        b = tc.Batch.from_edges([(r.src, r.dst, r.n) for r in group], stream=self.build_stream,
                                staging=self.staging)
        if self.params:
            b.set_params(**self.params)
        md = b.max_degree_vertices(stream=self.build_stream)
        return b, [md[i] if r.root is None else r.root for i, r in enumerate(group)]

    def count(self, batch, roots):
        return batch.count(roots, stream=self.count_stream)

    def release(self, batch) -> None:
        batch.close()


class Server:
    def __init__(self, hbm_budget_bytes: int = 64 << 30, max_batch: int = 4096, params=None,
                 backend=None):
        self.budget = int(hbm_budget_bytes)
        self.max_batch = max_batch
        self.backend = backend if backend is not None else GpuBackend(params)
        self.lock = threading.Condition()
        self.pending: deque = deque()     # arrived, not admitted
        self.ready: List = []             # (request, graph, root) built, waiting for a batch
        self.used = 0
        self.peak_used = 0
        self.completed: List[Request] = []
        self.batches: List[int] = []
        self.build_spans: List[tuple] = []   # (start, end) of each batch build, host clock
        self.count_spans: List[tuple] = []   # (start, end) of each batch count
        self.stopping = False
        self.threads = [threading.Thread(target=self._admit_loop, daemon=True),
                        threading.Thread(target=self._count_loop, daemon=True)]
        for t in self.threads:
            t.start()

    # -- client side ----------------------------------------------------------
    def submit(self, req: Request) -> Request:
        req.bytes = footprint_bytes(req.n, int(req.src.size))
        if req.bytes > self.budget:
            req.error = "request larger than the HBM budget"
            req.done = time.perf_counter()
            req.event.set()
            return req
        with self.lock:
            self.pending.append(req)
            self.lock.notify_all()
        return req

    def close(self) -> None:
        with self.lock:
            self.stopping = True
            self.lock.notify_all()
        for t in self.threads:
            t.join()

    # -- admission ------------------------------------------------------------
    def _admit_loop(self) -> None:
        while True:
            with self.lock:
                while not self.stopping and (not self.pending or
                                             self.used + self.pending[0].bytes > self.budget):
                    self.lock.wait(0.05)
                if self.stopping and not self.pending:
                    return
                group = []
                while (self.pending and len(group) < self.max_batch and
                       self.used + self.pending[0].bytes <= self.budget):
                    req = self.pending.popleft()
                    self.used += req.bytes
                    group.append(req)
                self.peak_used = max(self.peak_used, self.used)
            if not group:
                continue
            try:
                # one device build for the whole group: a batch straight from the edge lists
                t0 = time.perf_counter()
                b, roots = self.backend.build(group)
                t1 = time.perf_counter()
                with self.lock:
                    self.build_spans.append((t0, t1))
                    self.ready.append((group, b, roots))
                    self.lock.notify_all()
            except Exception as e:  # the group fails; its memory returns
                now = time.perf_counter()
                for r in group:
                    r.error, r.done = str(e), now
                    r.event.set()
                with self.lock:
                    self.used -= sum(r.bytes for r in group)
                    self.lock.notify_all()

    # -- counting -------------------------------------------------------------
    def _count_loop(self) -> None:
        while True:
            with self.lock:
                while not self.ready and not (self.stopping and not self.pending):
                    self.lock.wait(0.05)
                if not self.ready and self.stopping and not self.pending:
                    return
                reqs, b, roots = self.ready.pop(0)
            t0 = time.perf_counter()
            try:
                counts, err = self.backend.count(b, roots), None
            except Exception as e:
                counts, err = [None] * len(reqs), str(e)
            t1 = time.perf_counter()
            self.backend.release(b)
            now = time.perf_counter()
            for r, c in zip(reqs, counts):
                r.count, r.error, r.done = c, err, now
                r.event.set()
            with self.lock:
                self.used -= sum(r.bytes for r in reqs)
                self.completed.extend(reqs)
                self.batches.append(len(reqs))
                self.count_spans.append((t0, t1))
                self.lock.notify_all()

    # -- measurement ----------------------------------------------------------
    def overlap_stats(self) -> dict:
        """How much building and counting ran at the same time (host clock intervals).

        build_s / count_s: total time in batch builds / batch counts; overlap_s: the time in
        which a build and a count were both in progress; build_overlap_frac = overlap_s /
        build_s (1.0: every build ran while a count was on the device).
        """
        with self.lock:
            builds, counts = list(self.build_spans), list(self.count_spans)
        return overlap_of(builds, counts)


def overlap_of(builds, counts) -> dict:
    """Total lengths of two interval lists and of their intersection."""
    def merged(spans):
        out = []
        for a, b in sorted(spans):
            if out and a <= out[-1][1]:
                out[-1][1] = max(out[-1][1], b)
            else:
                out.append([a, b])
        return out
    mb, mc = merged(builds), merged(counts)
    i = j = 0
    both = 0.0
    while i < len(mb) and j < len(mc):
        lo, hi = max(mb[i][0], mc[j][0]), min(mb[i][1], mc[j][1])
        if hi > lo:
            both += hi - lo
        if mb[i][1] < mc[j][1]:
            i += 1
        else:
            j += 1
    build_s = sum(b - a for a, b in mb)
    count_s = sum(b - a for a, b in mc)
    return {"builds": len(builds), "counts": len(counts), "build_s": build_s,
            "count_s": count_s, "overlap_s": both,
            "build_overlap_frac": both / build_s if build_s > 0 else None}


def percentile(xs, q):
    if not xs:
        return None
    return float(np.percentile(np.asarray(xs), q))


def run_arrivals(server: Server, pool: list, rate: float, count: int, seed: int = 5,
                 big_every: int = 0, big_pool: Optional[list] = None) -> dict:
    """Poisson arrivals at `rate` graphs/s of `count` requests drawn from `pool`.

    A pool entry is ``(src, dst, n, root)``. With ``big_every`` = k, every k-th request is drawn from
    ``big_pool`` instead (the 1 % of large graphs). The call blocks until all requests have been
    answered.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    picks = rng.integers(0, len(pool), size=count)
    reqs = []
    t0 = time.perf_counter()
    next_t = t0
    for i in range(count):
        next_t += gaps[i]
        while True:
            now = time.perf_counter()
            if now >= next_t:
                break
            time.sleep(min(next_t - now, 0.002))
        use_big = big_every and big_pool and (i % big_every == big_every - 1)
        src, dst, n, root = (big_pool[i % len(big_pool)] if use_big else pool[picks[i]])
        r = Request(rid=i, src=src, dst=dst, n=n, root=root, arrival=time.perf_counter())
        reqs.append(server.submit(r))
    for r in reqs:
        r.event.wait()
    t1 = max(r.done for r in reqs)
    lat = [1e3 * r.latency() for r in reqs if r.error is None]
    return {"rate": rate, "requests": count, "errors": sum(r.error is not None for r in reqs),
            "seconds": t1 - t0, "graphs_per_s": count / (t1 - t0),
            "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
            "mean_ms": float(np.mean(lat)) if lat else None, "requests_list": reqs}
