"""Continuous-batching search server over one resident database.

Requests are single queries submitted at any time.  A dispatcher thread admits
pending requests into batches as device memory allows and plans each batch
(sw_queries_prepare, on a staging stream) while every stream slot may still
be busy, so that the next batch is planned by the time a slot frees up; it
then enqueues the batch's search (sw_search_prepared) and the copy of its
scores to pinned host memory on the free slot's CUDA stream, and completes
each request when its batch's event fires.  Batches on different streams
run concurrently, so the work of requests that arrive while others are on
the GPU overlaps on the device.

Every step of a search runs in libswgb.so; this module only schedules.
"""

import ctypes
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import _native as N
from .api import PreparedQueries, _mode


@dataclass(eq=False)
class Request:
    query: np.ndarray
    arrival: float
    future: Future
    admitted: float = 0.0
    planned: float = 0.0
    done: float = 0.0


@dataclass(eq=False)
class _Batch:
    requests: list
    prepared: PreparedQueries
    out_dev: object
    out_host: object
    event: object
    slot: int
    mem: int
    launched: float = field(default_factory=time.perf_counter)


class Server:
    """Continuous-batching server.

    db          a paper_2412_08308_gb300.api.Database
    submat      20x20 int8 scoring matrix; gap_open / gap_extend as in sw_search
    max_batch   most queries admitted into one batch
    n_streams   batches in flight at once (one CUDA stream each)
    mem_budget  device bytes the in-flight and planned batches may hold (scores, scratch)
    prestage    plan the next batch while no slot is free (False: plan when a
                slot frees up, on the critical path of the batch's requests)
    policy      "fifo" admits requests in arrival order; "sjf" admits the
                shortest queries first (their cells, query length x database,
                are the service time), except that a request waiting at least
                age_s seconds goes ahead of every younger one, oldest first
    """

    def __init__(self, db, submat, gap_open=10, gap_extend=2, mode="packed", max_batch=2, n_streams=2,
                 mem_budget=8 << 30, opts=None, policy="sjf", age_s=1.0, prestage=True):
        import torch

        self.torch = torch
        self.db = db
        self.submat = np.ascontiguousarray(submat, dtype=np.int8)
        self.gap_open, self.gap_extend, self.mode = int(gap_open), int(gap_extend), _mode(mode)
        self.max_batch = int(max_batch)
        self.mem_budget = int(mem_budget)
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        self.age_s = float(age_s)
        self.opts = opts
        self.streams = [torch.cuda.Stream() for _ in range(int(n_streams))]
        self.stage_stream = torch.cuda.Stream()
        self.prestage = bool(prestage)
        self.staged = None  # (requests, PreparedQueries, bytes): planned, waiting for a slot
        self.free_slots = list(range(len(self.streams)))
        self.pending = []
        self.inflight = []
        self.mem_used = 0
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self.stop = False
        self.completed = []
        self.cells = 0.0
        self.error = None
        self.thread = threading.Thread(target=self._run, name="swgb-serve", daemon=True)
        self.thread.start()

    # -- client side ---------------------------------------------------------
    def submit(self, query, arrival=None):
        fut = Future()
        q = np.ascontiguousarray(query, dtype=np.uint8)
        req = Request(q, time.perf_counter() if arrival is None else arrival, fut)
        with self.lock:
            if self.stop:
                raise RuntimeError("server closed")
            self.pending.append(req)
        self.wake.set()
        return fut

    def close(self):
        with self.lock:
            self.stop = True
        self.wake.set()
        self.thread.join()
        if self.error is not None:
            raise self.error

    # -- dispatcher ----------------------------------------------------------
    def _batch_bytes(self, reqs):
        n = self.db.n
        m = sum(len(r.query) for r in reqs)
        # scores (device + flags) + profile + a fixed allowance for the plan and boundary strips
        return len(reqs) * n * 8 + 21 * 4 * (m + 1024 * len(reqs)) + (256 << 20)

    def _order(self, now):
        """Pending requests in admission order."""
        if self.policy == "fifo":
            return list(self.pending)
        aged = [r for r in self.pending if now - r.arrival >= self.age_s]
        young = sorted((r for r in self.pending if now - r.arrival < self.age_s), key=lambda r: len(r.query))
        return aged + young

    def _stage(self):
        """Take the next batch from the pending requests and plan it (while
        the slots may still be busy, if prestage; else only with a slot free)."""
        with self.lock:
            if self.staged is not None or not self.pending:
                return False
            if not self.prestage and not self.free_slots:
                return False
            take = []
            for r in self._order(time.perf_counter()):
                if len(take) >= self.max_batch:
                    break
                if self.mem_used + self._batch_bytes(take + [r]) > self.mem_budget and take:
                    break
                take.append(r)
            need = self._batch_bytes(take)
            if self.mem_used + need > self.mem_budget and self.inflight:
                return False  # wait for memory to free up
            chosen = set(map(id, take))
            self.pending = [r for r in self.pending if id(r) not in chosen]
            self.mem_used += need
        now = time.perf_counter()
        for r in take:
            r.admitted = now
        lens = [len(r.query) for r in take]
        offsets = np.zeros(len(take) + 1, dtype=np.int64)
        offsets[1:] = np.cumsum(lens)
        residues = np.concatenate([r.query for r in take]) if offsets[-1] else np.zeros(0, np.uint8)
        with self.torch.cuda.stream(self.stage_stream):
            pq = PreparedQueries(self.db, residues, offsets, self.submat, self.gap_open, self.gap_extend,
                                 self.mode, opts=self.opts, stream=self.stage_stream)
        planned = time.perf_counter()
        for r in take:
            r.planned = planned
        self.staged = (take, pq, need)
        return True

    def _launch(self):
        """Enqueue the planned batch on a free slot's stream."""
        with self.lock:
            if self.staged is None or not self.free_slots:
                return False
            slot = self.free_slots.pop(0)
        take, pq, need = self.staged
        self.staged = None
        torch = self.torch
        stream = self.streams[slot]
        with torch.cuda.stream(stream):
            out_dev = torch.empty((len(take), self.db.n), dtype=torch.int32, device="cuda")
            out_host = torch.empty((len(take), self.db.n), dtype=torch.int32, pin_memory=True)
            pq.search(out_dev, stream=stream)
            out_host.copy_(out_dev, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.inflight.append(_Batch(take, pq, out_dev, out_host, ev, slot, need))
        self.cells += float(sum(len(r.query) for r in take)) * float(self.db.stats()[1])
        return True

    def _admit(self):
        """Launch what is planned, then plan the next batch; True if either happened."""
        launched = self._launch()
        staged = self._stage()
        if staged:
            launched = self._launch() or launched
        return launched or staged

    def _retire(self):
        done_any = False
        for b in list(self.inflight):
            if not b.event.query():
                continue
            rescued = N.sw_queries_status(b.prepared.handle, ctypes.c_void_p(self.streams[b.slot].cuda_stream))
            now = time.perf_counter()
            scores = b.out_host.numpy()
            for i, r in enumerate(b.requests):
                r.done = now
                r.future.set_result(scores[i].copy())
                self.completed.append(r)
            b.prepared.close()
            self.inflight.remove(b)
            with self.lock:
                self.free_slots.append(b.slot)
                self.mem_used -= b.mem
            done_any = True
            del rescued
        return done_any

    def _run(self):
        try:
            while True:
                progressed = self._retire()
                while self._admit():
                    progressed = True
                with self.lock:
                    finished = self.stop and not self.pending
                if finished and not self.inflight and self.staged is None:
                    return
                if not progressed:
                    self.wake.wait(timeout=0.0002)
                    self.wake.clear()
        except Exception as e:  # surface dispatcher failures to every waiter
            self.error = e
            with self.lock:
                waiting = self.pending + [r for b in self.inflight for r in b.requests]
                if self.staged is not None:
                    waiting += self.staged[0]
                self.pending = []
            for r in waiting:
                if not r.future.done():
                    r.future.set_exception(e)

    # -- statistics ----------------------------------------------------------
    def latency_stats(self):
        lat = np.array([r.done - r.arrival for r in self.completed])
        if lat.size == 0:
            return {}
        queue = np.array([r.admitted - r.arrival for r in self.completed])
        plan = np.array([r.planned - r.admitted for r in self.completed])
        p50 = float(np.percentile(lat, 50) * 1e3)
        # a request's latency = waiting for admission + planning its batch
        # (sw_queries_prepare, on the dispatcher thread) + its batch's search
        return {"requests": int(lat.size), "p50_ms": p50, "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "queue_ms_p50": float(np.median(queue) * 1e3),
                "plan_ms_p50": float(np.median(plan) * 1e3), "plan_ms_mean": float(plan.mean() * 1e3),
                "plan_share_of_p50": float(np.median(plan) * 1e3 / p50) if p50 > 0 else 0.0,
                "plan_share_of_mean": float(plan.mean() / lat.mean()) if lat.mean() > 0 else 0.0}
