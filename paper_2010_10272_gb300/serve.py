"""Serving loop: continuous batching of refinement requests on one GPU.

Requests (a hypergraph, a start partition, a round count) are queued as they arrive.  Each
tick of the server
  1. queues, on the batch stream, the next rounds of every resident request as one batch
     (hgp_batch_*: one launch per phase over all requests' work items): as many rounds as the
     request closest to completion still needs, so no request runs past its round count.  Up to
     `depth` ticks are queued on the device at once: the next tick's membership follows from
     the round counts alone, so it is queued before the previous tick's results are read, and
     the GPU does not wait for the host between ticks;
  2. while those rounds run on the GPU, admits queued requests: a request's state is created
     on the device (hgp_create, by a small pool of creator threads, each on its own upload
     stream, so creations overlap each other and the batch) if the memory budget minus what
     resident, staged and in-creation requests take covers its footprint estimate, so memory
     decides how many requests run at once; the new handles are staged and join the batch at
     the next tick (a round boundary);
  3. once the oldest queued tick has finished, reads its statistics (waiting for that tick
     only) and hands the requests it completed to a creator thread, which reads their
     partitions with one copy (hgp_batch_get_partitions), records their latency (arrival ->
     result on the host) and releases the tick's batch and their device state (queued behind
     the batch's rounds on each request's own stream, without synchronising the device).
Device memory comes from the library's stream-ordered pool, so creating and releasing request
state never synchronises the device.  Each request's arithmetic is the same as refining it
alone: batching changes only which kernel launch does the work (see tests/test_serving_gpu.py).
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import threading
import time
from typing import Deque, Dict, List, Optional

import numpy as np

from .native import HGP, Batch, set_blocking_waits

_RANGE = 256
_TILE = 2048
_BINS = 4096
_ALLOC_SLACK = 64 << 20
_DIRECT_TRANSPOSE_MAX_N = 1 << 21      # larger instances are transposed through bucketed pairs
_REORDER_MIN_NETS = 1 << 20            # from this many nets the handle keeps nets in internal order


def estimate_device_bytes(n: int, m: int, pins: int, k: int, max_net_size: int,
                          weighted_vertices: bool, weighted_nets: bool, subrounds: int = 4,
                          phi_width: int = 0) -> int:
    """Peak device bytes hgp_create needs for one hypergraph (mirrors its allocations)."""
    w = phi_width or (1 if max_net_size <= 255 else 2)
    n_ranges = (n + _RANGE - 1) // _RANGE
    n_tiles = (n_ranges + 7) // 8
    rec = 16 if k <= 32 else 32
    b = 0
    b += (m + 1) * 12 + pins * 8 + (n + 1) * 4 + n * 4 + n     # offsets, pins, inc, vtx_off, part
    b += n * 4 if weighted_vertices else 0
    b += m * 4 if weighted_nets else 0
    b += (m * k * w + 3) // 4 * 4 + m * rec                    # Phi, net records
    b += n_ranges * _RANGE * 9 + n_ranges * (subrounds + 1) * 2 + n_ranges * 4   # sub-round lists, candidates
    b += k * _BINS * 8 + k * n_tiles * 8 + 64 * 40             # approval scratch
    b += (max(n, m) + 1) * 4 + n * 4 + (m + 1) * 8            # creation temporaries
    if m >= _REORDER_MIN_NETS and max_net_size >= 8 * -(-pins // max(m, 1)):
        b += m * 4                                            # internal net order: input -> internal ids
    if n > _DIRECT_TRANSPOSE_MAX_N:
        b += pins * 8 + 3 * 4096 * 4                          # bucketed transpose: (vertex, net) pairs
    # each of the ~32 device allocations is rounded up to the allocator's 2 MiB granularity
    return int(b * 1.05) + _ALLOC_SLACK


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    m: int
    net_off: np.ndarray
    pins: np.ndarray
    k: int
    eps: float
    part: np.ndarray
    rounds: int
    vertex_w: Optional[np.ndarray] = None
    net_w: Optional[np.ndarray] = None
    subrounds: int = 4
    seed: int = 0
    max_net_size: Optional[int] = None    # largest net, if the producer knows it (else computed once)
    arrival: float = 0.0
    # filled by the server
    admitted: float = 0.0
    finished: float = 0.0
    result: Optional[np.ndarray] = None
    stats: Optional[np.ndarray] = None
    objective: int = 0

    @classmethod
    def from_hypergraph(cls, rid, hg, rounds=None, **kw):
        kw.setdefault("max_net_size", getattr(hg, "max_net_size", None))
        return cls(rid, hg.n, hg.m, hg.net_off, hg.pins, hg.k, hg.eps, hg.part,
                   hg.rounds if rounds is None else rounds, hg.vertex_w, hg.net_w, **kw)

    @property
    def num_pins(self) -> int:
        return int(self.net_off[-1])

    def footprint(self) -> int:
        """Device bytes the request's state needs (computed once; admission asks repeatedly)."""
        fp = getattr(self, "_footprint", None)
        if fp is None:
            if self.max_net_size is None:
                sizes = np.diff(self.net_off)
                self.max_net_size = int(sizes.max()) if sizes.size else 0
            fp = self._footprint = estimate_device_bytes(
                self.n, self.m, self.num_pins, self.k, self.max_net_size, self.vertex_w is not None,
                self.net_w is not None, self.subrounds)
        return fp

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Continuous-batching refinement server for one GPU (see the module docstring).

    memory_budget: device bytes the server may hold for requests (default: the free device
    memory when the server starts, minus reserve_bytes).  max_active: requests refined at once;
    max_staged: requests created (or being created) ahead of the batch they will join;
    creators: threads that create and retire request state (0: the serving thread itself);
    ctas_per_sm: persistent grid of the batch's gain and apply kernels (0: by occupancy; fewer
    leave room on each SM for the creations' kernels); depth: ticks queued on the device at once
    (1: each tick's results are read before the next is queued); blocking_waits: the library's
    host waits sleep instead of spinning (hgp_set_blocking_waits, process-wide), so that waiting
    creator threads leave the CPU to the others; tick_streams: streams the ticks take in turn
    (with depth >= 2, consecutive ticks then run concurrently and fill each other's launch gaps;
    a request in two ticks is ordered between them by the batches)."""

    def __init__(self, stream=None, reserve_bytes: int = 1 << 30,
                 memory_budget: Optional[int] = None, max_active: int = 1024, max_staged: int = 256,
                 graph: bool = False, creators: int = 8, ctas_per_sm: int = 0, join_at: int = 0,
                 depth: int = 2, blocking_waits: bool = False, tick_streams: int = 2,
                 clock=time.perf_counter):
        import torch
        self._torch = torch
        self.stream = stream
        self._tick_streams = [stream]
        if stream is not None:
            dev = torch.device("cuda", torch.cuda.current_device())
            self._tick_streams += [torch.cuda.Stream(dev) for _ in range(int(tick_streams) - 1)]
        self.reserve = int(reserve_bytes)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info()
            memory_budget = max(0, int(free) - self.reserve)
        self.memory_budget = int(memory_budget)
        self.max_active = int(max_active)
        self.max_staged = int(max_staged)
        self.graph = graph
        self.ctas_per_sm = int(ctas_per_sm)
        self.join_at = int(join_at)
        if depth < 1:
            raise ValueError("depth must be at least 1")
        self.depth = int(depth)
        if blocking_waits:
            set_blocking_waits(True)
        self.clock = clock
        self.queue: Deque[Request] = collections.deque()
        self.staged: Deque[Request] = collections.deque()
        self.active: List[Request] = []
        self._creating: Deque[tuple] = collections.deque()    # (request, future), FIFO
        self._retiring: Deque[tuple] = collections.deque()    # (request, future), FIFO
        self._handles: Dict[int, HGP] = {}
        self._planned: Dict[int, int] = {}                      # rounds queued per request
        self._stats: Dict[int, list] = {}
        # queued ticks, oldest first: (batch, members, rounds, members it completes)
        self._inflight: Deque[tuple] = collections.deque()
        self._resident_bytes = 0
        self._lock = threading.Lock()
        self._tls = threading.local()
        self._device = torch.cuda.current_device() if stream is not None else None
        self._pool = concurrent.futures.ThreadPoolExecutor(max_workers=creators) if creators > 0 else None
        self.ticks = 0
        self.rejected: List[Request] = []

    # -- requests
    def submit(self, req: Request, arrival: Optional[float] = None):
        req.arrival = self.clock() if arrival is None else arrival
        with self._lock:
            self.queue.append(req)

    def idle(self) -> bool:
        with self._lock:
            return (not self.queue and not self.active and not self.staged and not self._creating
                    and not self._retiring and not self._inflight)

    # -- admission by the memory budget
    def _free_bytes(self) -> int:
        return self.memory_budget - self._resident_bytes

    def _create(self, req: Request) -> HGP:
        """The request's device state, on the calling thread's upload stream."""
        stream = None
        if self.stream is not None:
            stream = getattr(self._tls, "stream", None)
            if stream is None:
                # high priority: a creation's short kernels go ahead of queued batch kernels
                self._torch.cuda.set_device(self._device)
                stream = self._tls.stream = self._torch.cuda.Stream(priority=-1)
        return HGP(req.n, req.m, req.net_off, req.pins, req.k, req.eps, req.part, req.vertex_w,
                   req.net_w, subrounds=req.subrounds, seed=req.seed, stream=stream)

    def _retire_group(self, batch, slots, reqs, handles):
        """The partitions of the requests a tick finished, read with one copy
        (hgp_batch_get_partitions), then the tick's batch and the requests' device state
        released (queued on each request's own stream, behind the batch)."""
        try:
            parts = batch.partitions(slots) if slots else [h.partition() for h in handles]
            now = self.clock()
            for req, part, h in zip(reqs, parts, handles):
                req.result = part
                req.finished = now
                req.objective = int(req.stats[-1][0]) if len(req.stats) else h.objective()
        finally:                                # released even when a read-back fails
            batch.close()
            for h in handles:
                h.close()

    def _install(self, req: Request, h: HGP):
        req.admitted = self.clock()
        self._handles[req.rid] = h
        self._planned[req.rid] = 0
        self._stats[req.rid] = []
        self.staged.append(req)

    def _admit(self):
        while len(self.staged) + len(self._creating) < self.max_staged:
            with self._lock:
                if not self.queue:
                    return
                req = self.queue[0]
            need = req.footprint()
            if need > self._free_bytes():
                if self._resident_bytes > 0:
                    return                      # wait for resident requests to finish
                with self._lock:                # larger than the whole budget: refuse it
                    self.queue.popleft()
                self.rejected.append(req)
                continue
            with self._lock:
                self.queue.popleft()
            self._resident_bytes += need
            req._bytes = need
            if self._pool is not None:
                self._creating.append((req, self._pool.submit(self._create, req)))
            else:
                self._install(req, self._create(req))

    def _collect(self, block: bool):
        """Stages the created requests, in admission order; with `block`, waits for the first."""
        while self._creating and (block or self._creating[0][1].done()):
            req, fut = self._creating.popleft()
            self._install(req, fut.result())
            block = False

    def _promote(self):
        # join_at: 0 = staged requests join at every round boundary; otherwise they join only
        # when at most join_at requests are still running (fewer, larger ticks)
        if self.join_at and len(self.active) > self.join_at:
            return
        while self.staged and len(self.active) < self.max_active:
            self.active.append(self.staged.popleft())

    def _can_launch(self) -> bool:
        return bool(self.active or self.staged) and len(self._inflight) < self.depth

    def _launch(self):
        """Queues the next rounds of the active requests as one batch call (no host wait)."""
        members = list(self.active)
        batch = Batch([self._handles[r.rid] for r in members], graph=self.graph,
                      stream=self._tick_streams[self.ticks % len(self._tick_streams)],
                      gain_ctas_per_sm=self.ctas_per_sm, apply_ctas_per_sm=self.ctas_per_sm)
        rounds = min(r.rounds - self._planned[r.rid] for r in members)
        if rounds:
            batch.refine(rounds, stats=False)
        self.ticks += 1
        finishing = []
        for r in members:
            self._planned[r.rid] += rounds
            if self._planned[r.rid] >= r.rounds:
                finishing.append(r)
        done_ids = {r.rid for r in finishing}
        self.active = [r for r in members if r.rid not in done_ids]
        self._inflight.append((batch, members, rounds, finishing))

    def _complete(self, tick):
        """Statistics of a finished (or the oldest) tick; its completed requests retire."""
        batch, members, rounds, finishing = tick
        if rounds:
            st = batch.stats(rounds)            # waits for this tick only
            for i, req in enumerate(members):
                self._stats[req.rid].extend(st[i])
        slot = {r.rid: i for i, r in enumerate(members)}
        slots = [slot[r.rid] for r in finishing] if rounds else []
        handles = [self._handles.pop(r.rid) for r in finishing]
        for req in finishing:
            req.stats = np.array(self._stats.pop(req.rid), dtype=np.int64)
            self._planned.pop(req.rid)
        if self._pool is not None and finishing:
            fut = self._pool.submit(self._retire_group, batch, slots, finishing, handles)
            for req in finishing:
                self._retiring.append((req, fut))
        else:
            self._retire_group(batch, slots, finishing, handles)
            for req in finishing:
                self._retiring.append((req, None))

    # -- one tick
    def step(self) -> List[Request]:
        """Let the staged requests join, queue the next rounds of the resident requests, admit
        arrivals while they run, and retire the requests of the oldest queued tick once it is
        done (or wait for it when no further tick can be queued)."""
        self._collect(block=False)
        self._promote()
        if self.active and len(self._inflight) < self.depth:
            self._launch()
        self._admit()
        if self._inflight and (not self._can_launch() or self._inflight[0][0].done()):
            self._complete(self._inflight.popleft())
        out = self._collect_retired(block=False)
        if out:
            self._admit()
        if not self._inflight and not self.active and not self.staged:
            if self._creating:
                self._collect(block=True)
            elif self._retiring:
                out.extend(self._collect_retired(block=True))
                self._admit()
        return out

    def _collect_retired(self, block: bool) -> List[Request]:
        """Requests whose results reached the host (their memory is free again), in order."""
        out = []
        while self._retiring and (block or self._retiring[0][1] is None or self._retiring[0][1].done()):
            req, fut = self._retiring.popleft()
            if fut is not None:
                fut.result()
            self._resident_bytes -= req._bytes
            out.append(req)
            block = False
        return out

    def run_until_idle(self) -> List[Request]:
        out = []
        while not self.idle():
            out.extend(self.step())
        return out

    def close(self):
        while self._creating:
            req, fut = self._creating.popleft()
            try:
                fut.result().close()
            except Exception:
                pass
        if self._pool is not None:
            self._pool.shutdown(wait=True)
        self._retiring.clear()
        while self._inflight:
            batch = self._inflight.popleft()[0]
            batch.synchronize()
            batch.close()
        for h in self._handles.values():
            h.close()
        self._handles.clear()


def latency_summary(reqs: List[Request]) -> dict:
    lat = np.array([r.latency for r in reqs], dtype=np.float64) * 1e3
    if lat.size == 0:
        return {"count": 0}
    return {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "max_ms": float(lat.max())}
