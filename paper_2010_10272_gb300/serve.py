"""Serving loop: continuous batching of refinement requests on one GPU.

Requests (a hypergraph, a start partition, a round count) are queued as they arrive.  Every
tick the server
  1. admits queued requests while the device has room for them: a request's state is created
     on the device (hgp_create) only if the free HBM minus a reserve covers its footprint
     estimate, so memory decides how many requests run at once;
  2. runs one LP round for every resident request in a single batch (hgp_batch_*: one launch
     per phase over all requests' work items), so requests that arrived while others were on
     the GPU share their kernels from the next round on;
  3. retires requests whose rounds are done: their partition is read back to the host, their
     device state is freed, and their latency (arrival -> result on the host) is recorded.
Each request's arithmetic is the same as refining it alone: batching changes only which
kernel launch does the work (see tests/test_serving_gpu.py).
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Deque, Dict, List, Optional

import numpy as np

from .native import HGP, Batch

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
    arrival: float = 0.0
    # filled by the server
    admitted: float = 0.0
    finished: float = 0.0
    result: Optional[np.ndarray] = None
    stats: Optional[np.ndarray] = None
    objective: int = 0

    @classmethod
    def from_hypergraph(cls, rid, hg, rounds=None, **kw):
        return cls(rid, hg.n, hg.m, hg.net_off, hg.pins, hg.k, hg.eps, hg.part,
                   hg.rounds if rounds is None else rounds, hg.vertex_w, hg.net_w, **kw)

    @property
    def num_pins(self) -> int:
        return int(self.net_off[-1])

    def footprint(self) -> int:
        sizes = np.diff(self.net_off)
        return estimate_device_bytes(self.n, self.m, self.num_pins, self.k,
                                     int(sizes.max()) if sizes.size else 0,
                                     self.vertex_w is not None, self.net_w is not None,
                                     self.subrounds)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Continuous-batching refinement server for one GPU (see the module docstring)."""

    def __init__(self, stream=None, reserve_bytes: int = 1 << 30,
                 memory_budget: Optional[int] = None, max_active: int = 1024, graph: bool = False,
                 clock=time.perf_counter):
        import torch
        self._torch = torch
        self.stream = stream
        self.reserve = int(reserve_bytes)
        self.memory_budget = memory_budget
        self.max_active = int(max_active)
        self.graph = graph
        self.clock = clock
        self.queue: Deque[Request] = collections.deque()
        self.active: List[Request] = []
        self._handles: Dict[int, HGP] = {}
        self._done_rounds: Dict[int, int] = {}
        self._stats: Dict[int, list] = {}
        self._batch: Optional[Batch] = None
        self._batch_key: tuple = ()
        self._resident_bytes = 0
        self._lock = threading.Lock()
        self.ticks = 0
        self.rejected: List[Request] = []

    # -- requests
    def submit(self, req: Request, arrival: Optional[float] = None):
        req.arrival = self.clock() if arrival is None else arrival
        with self._lock:
            self.queue.append(req)

    def idle(self) -> bool:
        with self._lock:
            return not self.queue and not self.active

    # -- admission by free HBM
    def _free_bytes(self) -> int:
        free, _ = self._torch.cuda.mem_get_info()
        if self.memory_budget is not None:
            free = min(free, self.memory_budget - self._resident_bytes)
        return free

    def _admit(self):
        while True:
            with self._lock:
                if not self.queue or len(self.active) >= self.max_active:
                    return
                req = self.queue[0]
            need = req.footprint()
            if need + self.reserve > self._free_bytes():
                if self.active:
                    return                      # wait for a resident request to finish
                if self.memory_budget is not None and need > self.memory_budget:
                    with self._lock:            # can never fit: refuse it
                        self.queue.popleft()
                    self.rejected.append(req)
                    continue
            with self._lock:
                self.queue.popleft()
            h = HGP(req.n, req.m, req.net_off, req.pins, req.k, req.eps, req.part, req.vertex_w,
                    req.net_w, subrounds=req.subrounds, seed=req.seed, stream=self.stream)
            req.admitted = self.clock()
            self._handles[req.rid] = h
            self._done_rounds[req.rid] = 0
            self._stats[req.rid] = []
            self._resident_bytes += need
            req._bytes = need
            self.active.append(req)

    # -- one tick
    def step(self) -> List[Request]:
        """Admit what fits, run one round for every resident request, retire finished ones."""
        self._admit()
        if not self.active:
            return []
        key = tuple(r.rid for r in self.active)
        if key != self._batch_key:
            if self._batch is not None:
                self._batch.close()
            self._batch = Batch([self._handles[rid] for rid in key], graph=self.graph,
                                stream=self.stream)
            self._batch_key = key
        st = self._batch.refine(1)
        self.ticks += 1
        finished = []
        for i, req in enumerate(self.active):
            self._stats[req.rid].append(st[i, 0])
            self._done_rounds[req.rid] += 1
            if self._done_rounds[req.rid] >= req.rounds:
                finished.append(req)
        if finished:
            done_ids = {r.rid for r in finished}
            keep = []
            for req in self.active:
                if req.rid in done_ids:
                    h = self._handles.pop(req.rid)
                    req.result = h.partition()
                    req.objective = h.objective()
                    req.stats = np.array(self._stats.pop(req.rid), dtype=np.int64)
                    req.finished = self.clock()
                    h.close()
                    self._done_rounds.pop(req.rid)
                    self._resident_bytes -= req._bytes
                else:
                    keep.append(req)
            self.active = keep
        return finished

    def run_until_idle(self) -> List[Request]:
        out = []
        while not self.idle():
            out.extend(self.step())
        return out

    def close(self):
        if self._batch is not None:
            self._batch.close()
            self._batch = None
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
