"""Serving loop: continuous batching of tree builds and query batches.

Build requests arrive over time.  At every step the server:
- retires the builds that have finished (their trees become resident and
  their latency, arrival to resident, is recorded);
- admits every queued request that fits the device-memory budget, evicting
  the oldest resident trees when that makes room;
- launches all admitted requests as one batched build (wt_build_batch) on the
  build stream.
Requests that arrive while a batch runs simply wait for the next step.
Query batches run on a second stream against the trees resident at the
time, through wt_query_multi, so queries and builds overlap on the device.
A tree is freed only after the query batches that may read it have
finished.  All device work happens in the library's kernels; this module
only schedules it.
"""
from __future__ import annotations

import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import wt as W


@dataclass
class BuildRequest:
    rid: int
    S: torch.Tensor | None   # device symbols (released once the tree is resident)
    sigma: int
    arrival: float           # host clock (time.perf_counter) when it arrived
    admitted: float = 0.0
    done: float = 0.0
    n: int = 0
    error: str | None = None  # why the request was rejected or its build failed


@dataclass
class QueryBatch:
    qid: int
    issued: float
    event: torch.cuda.Event
    out: torch.Tensor
    trees: list = field(default_factory=list)
    done: float = 0.0


def resident_bytes(n: int, sigma: int) -> int:
    """Device bytes a built tree of n symbols keeps: its bitmaps plus
    directories, about 1.07 n bits per level."""
    L = max(0, (sigma - 1).bit_length())
    return L * (n // 8 + n // 128 + n // 1024 + 4096)


def tree_bytes(n: int, sigma: int, width: int) -> int:
    """Device bytes a build of n symbols holds while it runs: the tree and
    its transient scratch (two order buffers, histogram and node tables)."""
    L = max(0, (sigma - 1).bit_length())
    scratch = 2 * n * width + (1 << L) * 32 + sigma * 8 + L * (n // 512 + 64)
    return resident_bytes(n, sigma) + scratch


class Server:
    def __init__(self, budget_bytes: int = 120 << 30, max_batch: int = 1024, device=None):
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.build_stream = torch.cuda.Stream(self.device)
        self.query_stream = torch.cuda.Stream(self.device)
        self.budget = budget_bytes
        self.max_batch = max_batch
        self.queue: deque[BuildRequest] = deque()
        self.inflight: list = []                  # (requests, trees, event)
        self.resident: OrderedDict = OrderedDict()  # rid -> (tree, bytes, request)
        self.used = 0
        self.peak_used = 0
        self.batch_host_ms: list[float] = []      # host time of each wt_build_batch call
        self.finished: list[BuildRequest] = []
        self.failed: list[BuildRequest] = []     # builds whose wait raised (their bytes are given back)
        self.rejected: list[BuildRequest] = []   # requests larger than the whole budget
        self.queries: list[QueryBatch] = []
        self.last_query_event: torch.cuda.Event | None = None
        self.evicted = 0
        self.built_symbols = 0
        self.batches = 0

    # ---------------------------------------------------------------- builds
    def submit(self, req: BuildRequest) -> None:
        self.queue.append(req)

    def _evict_oldest(self) -> bool:
        if not self.resident:
            return False
        rid, (tree, nbytes, req) = self.resident.popitem(last=False)
        if self.last_query_event is not None:
            # queries launched so far may read this tree: free after them
            self.build_stream.wait_event(self.last_query_event)
        with torch.cuda.stream(self.build_stream):
            tree.free()
        self.used -= nbytes
        self.evicted += 1
        return True

    def _admit(self) -> None:
        batch = []
        while self.queue and len(batch) < self.max_batch:
            req = self.queue[0]
            need = tree_bytes(req.S.numel(), req.sigma, req.S.element_size())
            if need > self.budget:
                # It can never fit: refuse it before evicting anything, so it
                # neither empties the resident set nor blocks the queue.
                self.queue.popleft()
                req.error = f"needs {need} bytes, more than the {self.budget}-byte budget"
                req.S = None
                self.rejected.append(req)
                continue
            while self.used + need > self.budget and self._evict_oldest():
                pass
            if self.used + need > self.budget:
                break
            self.queue.popleft()
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            req.admitted = time.perf_counter()
            batch.append((req, need))
        if not batch:
            return
        reqs = [r for r, _ in batch]
        self.build_stream.wait_stream(torch.cuda.current_stream(self.device))
        for r in reqs:
            r.S.record_stream(self.build_stream)
        h0 = time.perf_counter()
        trees = W.build_batch([r.S for r in reqs], [r.sigma for r in reqs], stream=self.build_stream, wait=False)
        self.batch_host_ms.append((time.perf_counter() - h0) * 1e3)
        ev = torch.cuda.Event()
        ev.record(self.build_stream)
        self.inflight.append((batch, trees, ev))
        self.batches += 1

    def _retire(self) -> None:
        still = []
        for batch, trees, ev in self.inflight:
            if not ev.query():
                still.append((batch, trees, ev))
                continue
            now = time.perf_counter()
            for (req, need), tree in zip(batch, trees):
                req.n = req.S.numel()
                req.S = None           # the build no longer reads it
                try:
                    tree.wait()        # raises if this sequence failed
                except W.WTError as e:
                    # Record the failure, give back its bytes and go on
                    # retiring the rest of the batch.
                    req.error = str(e)
                    self.failed.append(req)
                    self.used -= need
                    with torch.cuda.stream(self.build_stream):
                        tree.free()
                    continue
                req.done = now
                self.finished.append(req)
                # The build's scratch is freed: the tree keeps its own bytes.
                keep = resident_bytes(req.n, req.sigma)
                self.used -= need - keep
                self.resident[req.rid] = (tree, keep, req)
                self.built_symbols += req.n
        self.inflight = still

    def step(self) -> None:
        """Retire finished builds, then admit and launch what fits."""
        self._retire()
        self._admit()

    # --------------------------------------------------------------- queries
    def resident_trees(self) -> list:
        return [v[0] for v in self.resident.values()]

    def query(self, trees: list, tree_idx: torch.Tensor, op: torch.Tensor, c: torch.Tensor,
              arg: torch.Tensor) -> QueryBatch:
        """One batch of mixed queries on the query stream (inputs on the device)."""
        out = torch.empty(arg.numel(), dtype=torch.uint64, device=self.device)
        issued = time.perf_counter()
        self.query_stream.wait_stream(torch.cuda.current_stream(self.device))
        # The query stream reads tensors the caller's stream allocated: tell
        # the caching allocator, so their memory is not reused under it.
        for x in (tree_idx, op, c, arg, out):
            x.record_stream(self.query_stream)
        with torch.cuda.stream(self.query_stream):
            W.query_multi(trees, tree_idx, op, c, arg, out=out, stream=self.query_stream)
            ev = torch.cuda.Event()
            ev.record(self.query_stream)
        qb = QueryBatch(len(self.queries), issued, ev, out, trees)
        self.queries.append(qb)
        self.last_query_event = ev
        return qb

    def poll_queries(self) -> None:
        now = time.perf_counter()
        for qb in self.queries:
            if not qb.done and qb.event.query():
                qb.done = now
                qb.trees = []

    def drain(self) -> None:
        """Waits for every admitted build and query batch."""
        while self.queue or self.inflight:
            self.step()
            time.sleep(0.0001)
        torch.cuda.synchronize(self.device)
        self.poll_queries()

    def close(self) -> None:
        self.drain()
        torch.cuda.synchronize(self.device)
        for rid in list(self.resident):
            tree, nbytes, req = self.resident.pop(rid)
            tree.free()
        self.used = 0


def percentiles(xs, ps=(50, 99)):
    if len(xs) == 0:
        return {f"p{p}": None for p in ps}
    a = np.asarray(xs)
    return {f"p{p}": float(np.percentile(a, p)) for p in ps}
