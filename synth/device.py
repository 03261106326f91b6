"""Seeded serving-stream requests drawn on the GPU (torch's counter-based CUDA generator).

The serving benchmark needs thousands of distinct requests whose pin counts are log-uniform in
[10^4, 5*10^6] (about 8*10^5 pins on average), i.e. billions of pins per run: more than the
numpy generators of ``synth`` produce in the time the run should take.  This module draws the
same recipe as ``synth.serving_request`` (the planted model of ``synth.planted`` with
|e| = 2 + Poisson(4), p_in = 0.8, f = 0.3, n = m = ceil(P/6), k uniform in {2, 4, 8, 16, 32})
with torch on the device and returns host arrays in page-locked memory.  The random streams
differ from numpy's, so a request here is not the numpy request of the same seed; only the
distributions agree.  Like the rest of ``synth`` it holds random draws, sorting and CSR
assembly only.
"""
from __future__ import annotations

import math

import numpy as np

from . import Hypergraph

_KS = (2, 4, 8, 16, 32)


def serving_requests(seed: int, count: int, p_lo: int = 10_000, p_hi: int = 5_000_000,
                     device="cuda", pin_memory: bool = True):
    """`count` planted requests (``synth.Hypergraph``, 3 rounds each) drawn from one seed.

    All requests are drawn on the device first; their arrays are then copied into one host
    buffer (page-locked unless pin_memory is False) and returned as views into it, so the
    whole set costs one host allocation."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    hgen = np.random.Generator(np.random.PCG64(np.random.SeedSequence(int(seed))))
    drawn = []
    for i in range(count):
        P_target = math.exp(hgen.uniform(math.log(p_lo), math.log(p_hi)))
        n = int(math.ceil(P_target / 6.0))
        k = int(hgen.choice(_KS))
        arrs = _planted(gen, n, k, device)
        drawn.append((n, k, f"request[{i}] n=m={n} k={k}", arrs))
    # one host buffer for every array, each slice 8-byte aligned
    # largest net of each request (one device reduction per request, read back together)
    maxes = torch.stack([(a[0][1:] - a[0][:-1]).max() for _, _, _, a in drawn]).cpu().tolist() if drawn else []
    sizes = [[t.numel() * t.element_size() for t in arrs] for _, _, _, arrs in drawn]
    total = sum((b + 7) // 8 * 8 for row in sizes for b in row)
    buf = torch.empty(max(8, total), dtype=torch.uint8, pin_memory=pin_memory)
    out, off = [], 0
    views = []
    for (n, k, name, arrs), row in zip(drawn, sizes):
        host = []
        for t, b in zip(arrs, row):
            dst = buf[off:off + b]
            dst.copy_(t.view(torch.uint8).reshape(-1), non_blocking=True)
            host.append((off, b, t.dtype))
            off += (b + 7) // 8 * 8
        views.append((n, k, name, host))
    torch.cuda.synchronize() if str(device).startswith("cuda") else None
    base = buf.numpy()
    np_types = {torch.int64: np.int64, torch.int32: np.int32}
    for (n, k, name, host), mx in zip(views, maxes):
        a = [base[o:o + b].view(np_types[dt]) for o, b, dt in host]
        hg = Hypergraph(name, n, n, k, 0.03, a[0], a[1], a[2], None, None, 3)
        hg.max_net_size = int(mx)      # known from the draw; spares consumers a pass over net_off
        out.append(hg)
    del drawn
    return out


def _planted(gen, n: int, k: int, device, p_in: float = 0.8, f: float = 0.3, rate: float = 4.0):
    """Device arrays (net_off int64[m+1], pins int32[P], part int32[n]) of one planted
    request with m = n nets of size 2 + Poisson(rate) before de-duplication."""
    import torch
    m = n
    i64 = torch.int64
    perm = torch.randperm(n, generator=gen, device=device)
    group = torch.empty(n, dtype=i64, device=device)
    group[perm] = torch.arange(n, device=device) % k
    gsize = (n - torch.arange(k, device=device) + k - 1) // k
    sizes = 2 + torch.poisson(torch.full((m,), rate, device=device), generator=gen).to(i64)
    local = torch.repeat_interleave(torch.arange(m, device=device), sizes)
    P = local.numel()
    g = torch.randint(0, k, (m,), generator=gen, device=device)[local]
    in_group = torch.rand(P, generator=gen, device=device) < p_in
    member = (torch.rand(P, generator=gen, device=device, dtype=torch.float64) * gsize[g]).to(i64)
    member = torch.minimum(member, gsize[g] - 1)
    v_group = perm[g + k * member]
    v_unif = torch.randint(0, n, (P,), generator=gen, device=device)
    v = torch.where(in_group, v_group, v_unif)
    key = torch.unique(local * n + v)                       # sorted, duplicates dropped
    net = key // n
    pins = (key - net * n).to(torch.int32)
    cnt = torch.bincount(net, minlength=m)
    off = torch.zeros(m + 1, dtype=i64, device=device)
    torch.cumsum(cnt, 0, out=off[1:])
    part = group.clone()
    sel = torch.randperm(n, generator=gen, device=device)[: int(round(f * n))]
    part[sel] = torch.randint(0, k, (sel.numel(),), generator=gen, device=device)
    return off, pins, part.to(torch.int32)
