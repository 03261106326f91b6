"""Launch-shape autotuning for batches.

The persistent gain and apply kernels of a batch run on a grid of (CTAs per SM) x (SMs).
Results never depend on it; the best size depends on the batch (member sizes, k, record
layout).  tune_batch times hgp_batch_refine for each candidate on the batch's own handles and
returns the fastest.  Every trial starts from the handles' state at entry and the state is put
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
