"""Serving loop over a star schema resident in HBM: continuous batching of
select-join-group-by queries into shared scans.

The fact table is cut into ``segments`` row ranges.  Each GPU launch is one shared scan
(``crys_run_plans``) of the next segment for every active query, accumulating into the
queries' own outputs.  A query joins the circular scan at whatever segment comes next
and leaves after it has seen every segment once, so requests that arrive while others
are on the GPU start at the next launch instead of waiting for a batch to drain.
Admission: a query is admitted when one of the ``max_slots`` slots is free and its
hash tables plus outputs fit in ``memory_budget`` bytes next to the active queries';
its dimension tables are built (on the same stream) when it is admitted and released
when it completes.  Results are identical to running the query alone: integer sums,
every fact row counted exactly once.

With ``graphs=True`` (resident mode) every launch is a replay of a captured CUDA graph
(``ReplayedScan``): the host only writes the launch's argument block to pinned memory;
a query's outputs are cleared by its first launch and the batch is re-tagged only when
it changed.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import MAX_PLANS, check_device_errors
from .starschema import CompiledQuery, ReplayedScan, ResidentStarSchema


@dataclass
class Request:
    query: dict
    arrival_s: float
    admitted_s: float = -1.0
    done_s: float = -1.0
    result: tuple | None = None           # (sums, counts) numpy int64
    seen: int = 0
    compiled: CompiledQuery | None = None
    mem: int = 0
    deferred: bool = False

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class ServeStats:
    completed: int = 0
    wall_s: float = 0.0
    launches: int = 0
    deferred: int = 0
    max_active: int = 0
    replays: int = 0                      # launches that were CUDA graph replays
    h2d_bytes: int = 0                    # argument blocks copied from pinned host memory
    d2h_bytes: int = 0                    # results copied to pinned host memory
    peak_held_bytes: int = 0              # largest footprint of admitted + finishing queries
    latencies_s: list = field(default_factory=list)

    @property
    def qps(self) -> float:
        return self.completed / self.wall_s if self.wall_s > 0 else 0.0

    def percentile_ms(self, p: float) -> float:
        return float(np.percentile(np.array(self.latencies_s) * 1e3, p)) if self.latencies_s else 0.0


class QueryServer:
    def __init__(self, store: ResidentStarSchema, segments: int = 8, max_slots: int = MAX_PLANS,
                 memory_budget: int = 8 << 30, stream: torch.cuda.Stream | None = None,
                 mode: str = "resident", graphs: bool = True):
        if not 1 <= max_slots <= MAX_PLANS:
            raise ValueError("max_slots must be in 1..32")
        self.store = store
        self.mode = mode
        self.max_slots = max_slots
        self.memory_budget = memory_budget
        self.stream = stream or torch.cuda.Stream(device=store.device)
        n = store.n_rows
        step = -(-n // segments)
        step = (step + 4095) // 4096 * 4096           # segment starts stay 16-byte aligned
        self.bounds = [(b, min(n, b + step)) for b in range(0, n, step)] or [(0, 0)]
        self.next_segment = 0
        self.h2d_bytes = 0
        self.replay = ReplayedScan(store, self.stream) if graphs and mode == "resident" else None

    # -- admission ----------------------------------------------------------------------
    def fits(self, req: Request, active: list, finishing: tuple = ()) -> bool:
        """A free slot, and memory for `req` next to the active queries and the finishing
        ones whose last launch is still on the GPU (they hold their tables and outputs
        until that launch has been harvested)."""
        used = sum(r.mem for r in active) + sum(r.mem for r in finishing)
        return len(active) < self.max_slots and used + req.mem <= self.memory_budget

    def _admit(self, req: Request, now: float) -> None:
        with torch.cuda.stream(self.stream):
            req.compiled = self.store.compile(req.query, mode=self.mode, stream=self.stream,
                                              zero=self.replay is None)
        req.admitted_s = now
        req.seen = 0

    # -- one launch -------------------------------------------------------------------
    def _launch(self, active: list) -> None:
        b, e = self.bounds[self.next_segment]
        cqs = [r.compiled for r in active]
        fresh = [i for i, r in enumerate(active) if r.seen == 0]
        if self.replay is not None and self.replay.launch(cqs, b, e, fresh):
            self.h2d_bytes += self.replay.block_bytes
        else:
            with torch.cuda.stream(self.stream):
                if self.replay is not None:          # outputs were left for the replay to clear
                    for i in fresh:
                        cqs[i].sums.zero_()
                        cqs[i].counts.zero_()
                # outputs start at zero, so every launch accumulates
                self.store.run_shared(cqs, b, e, accumulate=True, stream=self.stream)
        for r in active:
            r.seen += 1
        self.next_segment = (self.next_segment + 1) % len(self.bounds)

    # -- driver -----------------------------------------------------------------------
    def prepare(self, queries: list, arrivals_s, realtime: bool = True) -> list:
        """Requests with their admission footprint; a query that could never be admitted
        (footprint above the whole budget) raises MemoryError before anything runs."""
        reqs = [Request(q, float(a) if realtime else 0.0) for q, a in zip(queries, arrivals_s)]
        for r in reqs:
            r.mem = self.store.memory_needed(r.query, self.mode)
            if r.mem > self.memory_budget:
                raise MemoryError(f"query {r.query.get('id')} needs {r.mem} B > budget "
                                  f"{self.memory_budget} B")
        return reqs

    def serve(self, queries: list, arrivals_s, realtime: bool = True) -> tuple:
        """Runs a request stream; returns (requests in input order, stats).

        With realtime=True requests become visible at their arrival time (seconds from
        the start); with realtime=False they are all queued at t=0 (closed loop)."""
        reqs = self.prepare(queries, arrivals_s, realtime)
        pending = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival_s)
        pi = 0
        active: list = []
        stats = ServeStats()
        nseg = len(self.bounds)
        self._sync()
        replays0 = self.replay.replays if self.replay is not None else 0
        self.h2d_bytes = 0
        t0 = time.perf_counter()
        inflight = None   # (event, finishing requests) of the launch on the GPU
        while pi < len(pending) or active or inflight:
            now = time.perf_counter() - t0
            while pi < len(pending) and reqs[pending[pi]].arrival_s <= now:
                r = reqs[pending[pi]]
                if not self.fits(r, active, inflight[1] if inflight else ()):
                    if not r.deferred:           # waits for a slot or memory to free up
                        r.deferred = True
                        stats.deferred += 1
                    break
                self._admit(r, now)
                active.append(r)
                pi += 1
            stats.max_active = max(stats.max_active, len(active))
            held = sum(r.mem for r in active) + (sum(r.mem for r in inflight[1]) if inflight else 0)
            stats.peak_held_bytes = max(stats.peak_held_bytes, held)
            if active:
                self._launch(active)
                stats.launches += 1
                finishing = [r for r in active if r.seen >= nseg]
                active = [r for r in active if r.seen < nseg]
                for r in finishing:
                    stats.d2h_bytes += self._copy_out(r)
                if inflight is not None:
                    self._harvest(inflight, t0, stats)
                inflight = (self._record(), finishing)
            else:
                if inflight is not None:
                    self._harvest(inflight, t0, stats)
                    inflight = None
                    continue
                if pi < len(pending):
                    wait = reqs[pending[pi]].arrival_s - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.001))
        stats.wall_s = time.perf_counter() - t0
        stats.replays = (self.replay.replays - replays0) if self.replay is not None else 0
        stats.h2d_bytes = self.h2d_bytes
        self._check()
        return reqs, stats

    # -- device plumbing (one place, so that the admission logic runs without a GPU) --------
    def _sync(self) -> None:
        torch.cuda.synchronize(self.store.device)

    def _record(self):
        ev = torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def _check(self) -> None:
        check_device_errors(self.stream)

    def _copy_out(self, r: Request) -> int:
        """Queues the copy of a finished query's sums and counts to pinned host memory on
        the serving stream; returns the bytes copied."""
        sums = torch.empty(r.compiled.groups, dtype=torch.int64, pin_memory=True)
        counts = torch.empty(r.compiled.groups, dtype=torch.int64, pin_memory=True)
        with torch.cuda.stream(self.stream):
            sums.copy_(r.compiled.sums, non_blocking=True)
            counts.copy_(r.compiled.counts, non_blocking=True)
        r.result = (sums, counts)
        return sums.numel() * sums.element_size() + counts.numel() * counts.element_size()

    def _harvest(self, inflight, t0, stats: ServeStats) -> None:
        ev, finishing = inflight
        ev.synchronize()
        done = time.perf_counter() - t0
        for r in finishing:
            r.done_s = done
            r.result = (r.result[0].numpy(), r.result[1].numpy())
            r.compiled = None                        # releases its hash tables and outputs
            stats.completed += 1
            stats.latencies_s.append(r.latency_s)


def one_at_a_time(store: ResidentStarSchema, queries: list, arrivals_s, realtime: bool = True,
                  stream=None, mode: str = "filtered"):
    """Baseline: FIFO, each query compiled and scanned alone (one fused probe kernel over
    all fact rows; by default the paper's plan with per-query filtered builds).  Returns
    (results, stats)."""
    stream = stream or torch.cuda.Stream(device=store.device)
    order = np.argsort(np.asarray(arrivals_s, dtype=np.float64), kind="stable")
    stats = ServeStats()
    results = [None] * len(queries)
    torch.cuda.synchronize(store.device)
    t0 = time.perf_counter()
    for i in order:
        arrival = float(arrivals_s[i]) if realtime else 0.0
        while realtime and time.perf_counter() - t0 < arrival:
            time.sleep(min(0.001, arrival - (time.perf_counter() - t0)))
        with torch.cuda.stream(stream):
            cq = store.compile(queries[i], mode=mode, stream=stream)
            store.run(cq, stream=stream)
            s = torch.empty(cq.groups, dtype=torch.int64, pin_memory=True)
            c = torch.empty(cq.groups, dtype=torch.int64, pin_memory=True)
            s.copy_(cq.sums, non_blocking=True)
            c.copy_(cq.counts, non_blocking=True)
        stream.synchronize()
        done = time.perf_counter() - t0
        results[i] = (s.numpy(), c.numpy())
        stats.completed += 1
        stats.latencies_s.append(done - arrival)
        stats.launches += 1
    stats.wall_s = time.perf_counter() - t0
    check_device_errors(stream)
    return results, stats
