"""Continuous-batching request loop over libvfunc (the serving pattern).

Requests arrive over time (e.g. Poisson): builds of a structure from host keys
and query batches against structures already built. The scheduler

* admits a build when its device-memory need fits the budget, and keeps it
  waiting otherwise, so builds enter as memory frees up;
* hands admitted builds to a build worker that builds small structures
  together with vf_build_batch and large ones alone with vf_build, on its own
  CUDA stream;
* hands queries whose structure is resident to a query worker that merges all
  of them into one vf_query_batch launch on another stream, so queries overlap
  with builds on the device;
* keeps finished structures resident on the device and records, per request,
  arrival, start and completion times (latency = completion - arrival).

Every call into the library releases the GIL (ctypes), so the two workers and
the scheduler run concurrently.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _binding as B


@dataclass
class BuildRequest:
    rid: int
    arrival: float           # seconds after the start of the run
    sid: int                 # structure id this build registers
    keys: torch.Tensor       # host int64 tensor holding uint64 keys (pinned preferred)
    values: torch.Tensor | None
    kind: int
    b: int
    seed: int


@dataclass
class QueryRequest:
    rid: int
    arrival: float
    sid: int
    keys: torch.Tensor       # host int64 tensor holding uint64 keys


@dataclass
class Record:
    rid: int
    kind: str
    arrival: float
    start: float = 0.0
    done: float = 0.0
    n: int = 0
    result: object = None

    @property
    def latency(self):
        return self.done - self.arrival


def build_need(n: int, b: int, fuse: bool) -> int:
    """Device bytes a build holds while it runs: keys, values, bucketed
    signatures/values, solver state and the data array."""
    data = int(n * 1.13 * b / 8) + 64
    per_key = 8 + 4 + 12 + (64 if fuse else 24)
    return n * per_key + data + (64 << 20)


def query_need(m: int) -> int:
    return 16 * m + (1 << 20)


@dataclass
class Server:
    device: int = 0
    budget: int = 8 << 30          # device bytes the loop may hold: in-flight work and resident arrays
    batch_below: int = 1 << 20     # builds smaller than this are batched together
    batch_keys: int = 1 << 26      # at most this many keys per batched build launch
    params: B.VfParams | None = None
    records: dict = field(default_factory=dict)
    resident: dict = field(default_factory=dict)

    def __post_init__(self):
        torch.cuda.set_device(self.device)
        self.params = self.params or B.vf_params_default()
        self.build_stream = torch.cuda.Stream(device=self.device)
        self.query_stream = torch.cuda.Stream(device=self.device)
        self._lock = threading.Condition()
        self._builds = collections.deque()     # admitted, not started
        self._queries = collections.deque()    # resident structure, not started
        self._in_use = 0       # accounted device bytes: admitted work plus resident data arrays
        self._inflight = 0     # admitted requests not yet finished
        self._stop = False
        self._errors = []

    # ------------------------------------------------------------------ workers
    def _now(self):
        return time.perf_counter() - self._t0

    def _build_worker(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._lock:
                while not self._builds and not self._stop:
                    self._lock.wait(0.01)
                if self._stop and not self._builds:
                    return
                batch, keys = [], 0
                while self._builds:
                    r = self._builds[0]
                    if batch and (len(r.keys) >= self.batch_below or keys + len(r.keys) > self.batch_keys):
                        break
                    batch.append(self._builds.popleft())
                    keys += len(r.keys)
                    if len(r.keys) >= self.batch_below:
                        break
            try:
                self._run_builds(batch)
            except Exception as e:  # recorded and re-raised by run()
                self._errors.append(e)
                with self._lock:
                    self._stop = True
                    self._lock.notify_all()
                return

    def _run_builds(self, batch):
        t = self._now()
        for r in batch:
            self.records[r.rid].start = t
        with torch.cuda.stream(self.build_stream):
            dev = [(r.keys.to(self.device, non_blocking=True),
                    None if r.values is None else r.values.to(self.device, non_blocking=True)) for r in batch]
            if len(batch) == 1 and len(batch[0].keys) >= self.batch_below:
                r = batch[0]
                p = B.vf_params_default(kind=r.kind, b=r.b, seed=r.seed)
                structs = [B.vf_build(dev[0][0], dev[0][1], params=p, stream=self.build_stream)]
            else:
                items = [(k, v, r.kind, r.b, r.seed) for (k, v), r in zip(dev, batch)]
                structs = B.vf_build_batch(items, params=self.params, stream=self.build_stream)
            self.build_stream.synchronize()
        done = self._now()
        with self._lock:
            for r, s in zip(batch, structs):
                rec = self.records[r.rid]
                rec.done = done
                rec.result = s.info
                self.resident[r.sid] = s
                info = s.info
                self._in_use -= build_need(len(r.keys), r.b, info.regime == B.REGIME_FUSE) - int(info.data_bytes)
                self._inflight -= 1
            self._lock.notify_all()

    def _query_worker(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._lock:
                while not self._queries and not self._stop:
                    self._lock.wait(0.01)
                if self._stop and not self._queries:
                    return
                batch = list(self._queries)
                self._queries.clear()
            try:
                self._run_queries(batch)
            except Exception as e:
                self._errors.append(e)
                with self._lock:
                    self._stop = True
                    self._lock.notify_all()
                return

    def _run_queries(self, batch):
        t = self._now()
        for r in batch:
            self.records[r.rid].start = t
        with torch.cuda.stream(self.query_stream):
            reqs = [(self.resident[r.sid], r.keys.to(self.device, non_blocking=True), None) for r in batch]
            outs = B.vf_query_batch(reqs, stream=self.query_stream)
            host = [o.to("cpu", non_blocking=True) for o in outs]
            self.query_stream.synchronize()
        done = self._now()
        with self._lock:
            for r, h in zip(batch, host):
                rec = self.records[r.rid]
                rec.done = done
                rec.result = h
                self._in_use -= query_need(len(r.keys))
                self._inflight -= 1
            self._lock.notify_all()

    # ------------------------------------------------------------------ scheduler
    def run(self, requests, realtime: bool = True):
        """Serve `requests` (sorted by arrival). Returns the per-request records."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            self.records[r.rid] = Record(r.rid, "build" if isinstance(r, BuildRequest) else "query", r.arrival,
                                         n=len(r.keys))
        waiting_b, waiting_q = collections.deque(), collections.deque()
        self._t0 = time.perf_counter()
        workers = [threading.Thread(target=self._build_worker, daemon=True),
                   threading.Thread(target=self._query_worker, daemon=True)]
        for w in workers:
            w.start()
        i = 0
        try:
            while True:
                now = self._now()
                while i < len(reqs) and (reqs[i].arrival <= now or not realtime):
                    (waiting_b if isinstance(reqs[i], BuildRequest) else waiting_q).append(reqs[i])
                    i += 1
                with self._lock:
                    if self._errors:
                        break
                    # builds: in arrival order while memory allows; one that does not fit
                    # (beyond the budget, or with resident arrays filling it) runs once
                    # nothing else is in flight
                    while waiting_b:
                        r = waiting_b[0]
                        need = build_need(len(r.keys), r.b, len(r.keys) >= self.params.lge_threshold)
                        if self._in_use + need > self.budget and self._inflight > 0:
                            break
                        self._in_use += need
                        self._inflight += 1
                        self._builds.append(waiting_b.popleft())
                    # queries: once their structure is resident and memory allows
                    keep = collections.deque()
                    while waiting_q:
                        r = waiting_q.popleft()
                        need = query_need(len(r.keys))
                        if r.sid in self.resident and (self._in_use + need <= self.budget or self._inflight == 0):
                            self._in_use += need
                            self._inflight += 1
                            self._queries.append(r)
                        else:
                            keep.append(r)
                    waiting_q = keep
                    self._lock.notify_all()
                    finished = all(rec.done > 0 for rec in self.records.values())
                if finished:
                    break
                time.sleep(0.0002)
        finally:
            with self._lock:
                self._stop = True
                self._lock.notify_all()
            for w in workers:
                w.join()
        if self._errors:
            raise self._errors[0]
        return self.records

    def close(self):
        for s in self.resident.values():
            s.free()
        self.resident.clear()


def percentiles(records, kind):
    lat = np.array([r.latency for r in records.values() if r.kind == kind])
    if len(lat) == 0:
        return {"n": 0}
    return {"n": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}
