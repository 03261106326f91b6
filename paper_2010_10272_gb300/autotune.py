"""Autotuning of the choices that do not change results.

* Launch shape: the persistent gain and apply kernels run on a grid of (CTAs per SM) x (SMs);
  the best size depends on the instance or batch (sizes, k, record layout).
* Phi entry width: 1, 2 or 4 bytes per entry (nets beyond the width's range keep int32 rows in
  the wide table); narrower rows halve the table and its initialisation, wider ones put fewer
  nets in the wide table.

tune_batch times hgp_batch_refine for each launch-shape candidate on the batch's own handles;
tune_instance creates the instance once per candidate width (timing the creation) and times
refinement for each launch shape.  Every trial starts from the same state and the state is put
back afterwards (hgp_export_state / hgp_import_state), so tuning changes nothing a later call
computes.
"""
from __future__ import annotations

from typing import Iterable, Optional, Sequence, Tuple

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = ((0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (2, 4), (4, 2))


def tune_batch(handles: Sequence, rounds: int = 1, candidates: Optional[Iterable[Tuple[int, int]]] = None,
               repeats: int = 2, stream=None) -> dict:
    """Returns {"gain_ctas_per_sm": g, "apply_ctas_per_sm": a, "ms": {(g, a): best ms}}.

    handles: HGP objects on the current device (the batch is built and destroyed here for
    every candidate); rounds: rounds per timed call; (0, 0) means occupancy-derived grids."""
    import torch
    from .native import Batch

    cands = list(candidates or DEFAULT_CANDIDATES)
    saved = [h.export_state() for h in handles]
    st = stream if stream is not None else torch.cuda.current_stream()
    times = {}
    try:
        for g, a in cands:
            b = Batch(handles, graph=True, gain_ctas_per_sm=g, apply_ctas_per_sm=a, stream=st)
            best = float("inf")
            for rep in range(repeats + 1):         # the first call captures the graph
                for h, s in zip(handles, saved):
                    h.import_state(s)
                torch.cuda.synchronize()
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(st)
                b.refine(rounds, stats=False)
                ev[1].record(st)
                torch.cuda.synchronize()
                if rep > 0:
                    best = min(best, ev[0].elapsed_time(ev[1]))
            b.close()
            times[(g, a)] = best
    finally:
        for h, s in zip(handles, saved):
            h.import_state(s)
        torch.cuda.synchronize()
    g, a = min(times, key=times.get)
    return {"gain_ctas_per_sm": g, "apply_ctas_per_sm": a, "ms": times}


def tune_instance(n, m, net_off, pins, k, eps, part, vertex_w=None, net_w=None, rounds: int = 1,
                  widths: Iterable[int] = (1, 2), shapes: Optional[Iterable[Tuple[int, int]]] = None,
                  repeats: int = 2, subrounds: int = 4, seed: int = 0, stream=None) -> dict:
    """Best (phi_width, gain_ctas_per_sm, apply_ctas_per_sm) for one instance by the time of a
    creation plus `rounds` rounds.  Arrays are torch CUDA tensors (device=True creation).
    Returns {"phi_width": w, "gain_ctas_per_sm": g, "apply_ctas_per_sm": a, "create_ms": {w: ms},
    "refine_ms": {(w, g, a): ms}}."""
    import time
    import torch
    from .native import HGP

    st = stream if stream is not None else torch.cuda.current_stream()
    cands = list(shapes or DEFAULT_CANDIDATES)
    create_ms, refine_ms = {}, {}
    for w in widths:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = HGP(n, m, net_off, pins, k, eps, part, vertex_w, net_w, subrounds=subrounds, seed=seed,
                phi_width=w, device=True, stream=st)
        torch.cuda.synchronize()
        create_ms[w] = (time.perf_counter() - t0) * 1e3
        w_eff = h.info()["phi_width"]
        saved = h.export_state()
        for g, a in cands:
            h.set_launch_shape(g, a)
            best = float("inf")
            for rep in range(repeats + 1):
                h.import_state(saved)
                torch.cuda.synchronize()
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(st)
                h.refine(rounds, stats=False)
                ev[1].record(st)
                torch.cuda.synchronize()
                if rep > 0:
                    best = min(best, ev[0].elapsed_time(ev[1]))
            refine_ms[(w_eff, g, a)] = best
        h.close()
        if w != w_eff:
            create_ms[w_eff] = create_ms.pop(w)
    w, g, a = min(refine_ms, key=lambda key: refine_ms[key] + create_ms[key[0]] / max(1, rounds))
    return {"phi_width": w, "gain_ctas_per_sm": g, "apply_ctas_per_sm": a, "create_ms": create_ms,
            "refine_ms": refine_ms}
