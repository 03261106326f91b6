"""Seeded synthetic hypergraph generators.

These produce the inputs that both the CUDA path and the CPU oracle consume.  They
contain none of the refinement arithmetic: only random draws, sorting and CSR
assembly.  Every generator is driven by ``numpy.random.Generator(PCG64(SeedSequence))``
and is deterministic for a given seed on any machine.

The instances stand in for the benchmark sets of the paper (SuiteSparse row-net
matrices, SAT and VLSI hypergraphs, Sec. 7 "Instances"), which are not available here.
Recipes:

* ``planted``: hidden group of v = (rank of v in a seeded permutation) mod k, so the
  groups are exactly balanced.  Each net draws a group uniformly; each of its pins is
  a uniform member of that group with probability ``p_in``, else a uniform vertex.
  Pins inside a net are sorted and de-duplicated, so a drawn size is an upper bound.
  Start partition: the hidden groups, then a fraction ``f`` of the vertices (sampled
  without replacement) reassigned to uniform blocks.
* ``rownet``: the row-net model of a random sparse matrix: row i is a net, columns are
  vertices; a row holds 1+Poisson(9) non-zeros, each at column (i + U{-5000..5000})
  mod n_cols with probability 0.7, else a uniform column.  Start: rank mod k.

Named configurations (sizes and distributions of the benchmark workloads):

* ``config_small``     n=m=10^4, k=2, |e|=2+Poisson(4), p_in=0.8, f=0.3, 5 rounds.
* ``config_rownet``    2*10^6 x 2*10^6 row-net, k=8, 10 rounds.
* ``config_batch``     256 planted instances, n log-uniform in [10^3, 2*10^5],
                       |e|=min(2+Zipf(2.5), 1000), k in {2,4,8,16}, c(v) in U{1..4}.
* ``config_powerlaw``  n=m=5*10^7, |e|=min(2+Zipf(2.1), 10^5), k=64, omega in U{1..10},
                       p_in=0.6, f=0.4, 5 rounds.
* ``serving_request``  planted, pins log-uniform in [10^4, 5*10^6], |e|=2+Poisson(4),
                       n=m=ceil(P/6), k in {2,4,8,16,32}, 3 rounds.

All accept ``scale`` (0 < scale <= 1) to draw a proportionally smaller instance with
the same distributions, used for quick tests and bounded CPU samples.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# nets are generated in fixed-size chunks; the chunk size is part of the recipe
# (it fixes the order in which random numbers are drawn)
_CHUNK_NETS = 1 << 20


@dataclasses.dataclass
class Hypergraph:
    """A weighted hypergraph H=(V,E,c,omega) in net->pins CSR form plus a start partition."""
    name: str
    n: int
    m: int
    k: int
    eps: float
    net_off: np.ndarray            # int64 [m+1]
    pins: np.ndarray               # int32 [P]
    part: np.ndarray               # int32 [n], start partition, values in [0, k)
    vertex_w: Optional[np.ndarray] = None   # int32 [n] or None (unit)
    net_w: Optional[np.ndarray] = None      # int32 [m] or None (unit)
    rounds: int = 5

    @property
    def num_pins(self) -> int:
        return int(self.net_off[-1])

    def net_sizes(self) -> np.ndarray:
        return np.diff(self.net_off)

    def total_vertex_weight(self) -> int:
        return int(self.n if self.vertex_w is None else self.vertex_w.astype(np.int64).sum())


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.SeedSequence):
        return np.random.Generator(np.random.PCG64(seed))
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))


def _dedup_chunk(local_net: np.ndarray, v: np.ndarray, n: int, count: int):
    """Sort pins inside each net and drop duplicates; returns (sizes[count], pins)."""
    key = local_net.astype(np.int64) * n + v.astype(np.int64)
    key.sort(kind="stable")
    if key.size:
        keep = np.empty(key.size, dtype=bool)
        keep[0] = True
        np.not_equal(key[1:], key[:-1], out=keep[1:])
        key = key[keep]
    nets = key // n
    sizes = np.bincount(nets, minlength=count).astype(np.int64)
    return sizes, (key - nets * n).astype(np.int32)


def _assemble(size_chunks, pin_chunks, m):
    sizes = np.concatenate(size_chunks) if size_chunks else np.zeros(0, np.int64)
    off = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    pins = np.concatenate(pin_chunks) if pin_chunks else np.zeros(0, np.int32)
    return off, pins


def hidden_groups(rng: np.random.Generator, n: int, k: int):
    """Group of v = rank of v in a seeded permutation, mod k.  Returns (perm, group)."""
    perm = rng.permutation(n)
    group = np.empty(n, dtype=np.int32)
    group[perm] = (np.arange(n, dtype=np.int64) % k).astype(np.int32)
    return perm, group


def perturb(rng: np.random.Generator, part: np.ndarray, k: int, f: float) -> np.ndarray:
    """Reassign round(f*n) vertices, sampled without replacement, to uniform blocks."""
    part = part.copy()
    cnt = int(round(f * part.size))
    if cnt:
        sel = rng.choice(part.size, size=cnt, replace=False)
        part[sel] = rng.integers(0, k, size=cnt, dtype=np.int32)
    return part


def planted(seed, n: int, m: int, k: int, size_fn, p_in: float, f: float,
            eps: float = 0.03, rounds: int = 5, vertex_w_max: int = 0,
            net_w_max: int = 0, name: str = "planted") -> Hypergraph:
    """Planted-partition hypergraph (recipe in the module docstring).

    ``size_fn(rng, count) -> int64 array`` draws net sizes; ``vertex_w_max``/``net_w_max``
    > 0 draw integer weights uniform in [1, max], 0 means unit weights.
    """
    rng = _rng(seed)
    perm, group = hidden_groups(rng, n, k)
    gsize = np.array([(n - g + k - 1) // k for g in range(k)], dtype=np.int64)
    size_chunks, pin_chunks = [], []
    for a in range(0, m, _CHUNK_NETS):
        b = min(m, a + _CHUNK_NETS)
        cnt = b - a
        sizes = np.asarray(size_fn(rng, cnt), dtype=np.int64)
        ngroup = rng.integers(0, k, size=cnt)
        local = np.repeat(np.arange(cnt, dtype=np.int64), sizes)
        g = ngroup[local]
        P = local.size
        in_group = rng.random(P) < p_in
        member = rng.integers(0, gsize[g])                 # index inside group g
        v_group = perm[g + k * member]
        v_unif = rng.integers(0, n, size=P)
        v = np.where(in_group, v_group, v_unif)
        s, p = _dedup_chunk(local, v, n, cnt)
        size_chunks.append(s)
        pin_chunks.append(p)
    off, pins = _assemble(size_chunks, pin_chunks, m)
    part = perturb(rng, group, k, f)
    vw = rng.integers(1, vertex_w_max + 1, size=n, dtype=np.int32) if vertex_w_max > 0 else None
    nw = rng.integers(1, net_w_max + 1, size=m, dtype=np.int32) if net_w_max > 0 else None
    return Hypergraph(name, n, m, k, eps, off, pins, part.astype(np.int32), vw, nw, rounds)


def rownet(seed, n_rows: int, n_cols: int, k: int, mean_extra: float = 9.0,
           band: int = 5000, p_band: float = 0.7, eps: float = 0.03, rounds: int = 10,
           name: str = "rownet") -> Hypergraph:
    """Row-net hypergraph of a random banded sparse matrix (module docstring)."""
    rng = _rng(seed)
    size_chunks, pin_chunks = [], []
    for a in range(0, n_rows, _CHUNK_NETS):
        b = min(n_rows, a + _CHUNK_NETS)
        cnt = b - a
        sizes = 1 + rng.poisson(mean_extra, size=cnt).astype(np.int64)
        local = np.repeat(np.arange(cnt, dtype=np.int64), sizes)
        row = local + a
        P = local.size
        banded = rng.random(P) < p_band
        off = rng.integers(-band, band + 1, size=P)
        v_band = np.mod(row + off, n_cols)
        v_unif = rng.integers(0, n_cols, size=P)
        v = np.where(banded, v_band, v_unif)
        s, p = _dedup_chunk(local, v, n_cols, cnt)
        size_chunks.append(s)
        pin_chunks.append(p)
    off, pins = _assemble(size_chunks, pin_chunks, n_rows)
    perm = rng.permutation(n_cols)
    part = np.empty(n_cols, dtype=np.int32)
    part[perm] = (np.arange(n_cols, dtype=np.int64) % k).astype(np.int32)
    return Hypergraph(name, n_cols, n_rows, k, eps, off, pins, part, None, None, rounds)


def poisson_sizes(lam: float, base: int = 2):
    def fn(rng, cnt):
        return base + rng.poisson(lam, size=cnt).astype(np.int64)
    return fn


def zipf_sizes(a: float, cap: int, base: int = 2):
    """Net size min(base + Zipf(a), cap)."""
    def fn(rng, cnt):
        z = rng.zipf(a, size=cnt).astype(np.float64)
        return np.minimum(base + z, cap).astype(np.int64)
    return fn


def _scaled(x: int, scale: float, lo: int = 16) -> int:
    return max(lo, int(round(x * scale)))


def config_small(scale: float = 1.0, seed: int = 1) -> Hypergraph:
    n = _scaled(10_000, scale)
    return planted(seed, n, n, 2, poisson_sizes(4.0), 0.8, 0.3, rounds=5,
                   name=f"planted n=m={n} k=2 |e|=2+Poisson(4)")


def config_rownet(scale: float = 1.0, seed: int = 1) -> Hypergraph:
    n = _scaled(2_000_000, scale)
    band = max(1, int(round(5000 * min(1.0, scale * 4))))
    return rownet(seed, n, n, 8, band=band, rounds=10,
                  name=f"row-net {n}x{n} nnz/row=1+Poisson(9) band=+-{band} k=8")


def config_powerlaw(scale: float = 1.0, seed: int = 1, cap: int = 100_000) -> Hypergraph:
    n = _scaled(50_000_000, scale)
    return planted(seed, n, n, 64, zipf_sizes(2.1, cap), 0.6, 0.4, rounds=5,
                   net_w_max=10,
                   name=f"power-law n=m={n} |e|=min(2+Zipf(2.1),{cap}) k=64 omega=U{{1..10}}")


def config_batch(count: int = 256, seed: int = 1, n_lo: int = 1_000,
                 n_hi: int = 200_000) -> List[Hypergraph]:
    """Uneven batch: each child seed draws n log-uniform, k, and the instance."""
    children = np.random.SeedSequence(seed).spawn(count)
    out = []
    for i, ss in enumerate(children):
        rng = _rng(ss.spawn(1)[0])
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        k = int(rng.choice([2, 4, 8, 16]))
        out.append(planted(ss, n, n, k, zipf_sizes(2.5, 1000), 0.8, 0.3, rounds=5,
                           vertex_w_max=4, name=f"batch[{i}] n=m={n} k={k}"))
    return out


def serving_request(seed, p_lo: int = 10_000, p_hi: int = 5_000_000) -> Hypergraph:
    """One serving request: a planted hypergraph with log-uniform pin count."""
    rng = _rng(seed)
    P = math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))
    n = int(math.ceil(P / 6.0))
    k = int(rng.choice([2, 4, 8, 16, 32]))
    sub = np.random.SeedSequence(int(rng.integers(0, 2**63 - 1)))
    return planted(sub, n, n, k, poisson_sizes(4.0), 0.8, 0.3, rounds=3,
                   name=f"request n=m={n} k={k}")


def random_small(seed, n: int, m: int, k: int, max_size: int = 6, weighted: bool = False,
                 p_in: float = 0.7, f: float = 0.5, eps: float = 0.03, rounds: int = 3):
    """Small planted instance with optional vertex/net weights, for unit and parity tests."""
    def fn(rng, cnt):
        return rng.integers(1, max_size + 1, size=cnt).astype(np.int64)
    return planted(seed, n, m, k, fn, p_in, f, eps=eps, rounds=rounds,
                   vertex_w_max=5 if weighted else 0, net_w_max=7 if weighted else 0,
                   name=f"random n={n} m={m} k={k}")
