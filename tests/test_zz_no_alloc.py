"""Allocation-free gain step (hgp_candidates_noalloc) against the allocating entry point.

Callers that cannot allocate device memory (an application allocator owning the device,
host callbacks where cudaMalloc is not allowed, paths that must not block on the allocator)
use hgp_candidates_noalloc, whose only scratch is a fixed array inside the library.  Its
output must equal hgp_debug_candidates on a freshly created handle, on two calls in a row
(the second call reuses the scratch the first one left behind).  This file is collected
last on purpose.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _transpose(hg):
    sizes = np.diff(hg.net_off)
    net_of_pin = np.repeat(np.arange(hg.m, dtype=np.int32), sizes)
    order = np.argsort(hg.pins, kind="stable")
    inc = net_of_pin[order].astype(np.int32)
    deg = np.bincount(hg.pins, minlength=hg.n)
    vtx_off = np.zeros(hg.n + 1, dtype=np.int32)
    vtx_off[1:] = np.cumsum(deg)
    return vtx_off, inc


@pytest.mark.parametrize("k,weighted,S", [(8, True, 4), (64, True, 3), (2, False, 2)])
def test_noalloc_matches_allocating_entry_point(k, weighted, S):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import HGP, build
    from paper_2010_10272_gb300.native import candidates_noalloc
    build.build()
    hg = synth.random_small(900 + k, 12000, 10000, k, max_size=9, weighted=weighted)
    vtx_off, inc = _transpose(hg)
    dev = torch.device("cuda:0")
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    args = [t(hg.net_off.astype(np.int32)), t(hg.pins), t(vtx_off), t(inc)]
    target = torch.empty(hg.n, dtype=torch.int32, device=dev)
    gain = torch.empty(hg.n, dtype=torch.int64, device=dev)
    h = HGP.from_hypergraph(hg, subrounds=S, seed=7)
    for s in (0, 1):                       # two calls in a row share the scratch array
        rc = candidates_noalloc(hg.n, hg.m, *args, hg.k, hg.eps, t(hg.part), target, gain,
                                vertex_w=t(hg.vertex_w), net_w=t(hg.net_w), subrounds=S, seed=7, s=s)
        assert rc == 0
        torch.cuda.synchronize()
        want_t, want_g = h.debug_candidates(s)
        np.testing.assert_array_equal(target.cpu().numpy(), want_t)
        np.testing.assert_array_equal(gain.cpu().numpy(), want_g)
        assert (want_t >= 0).any()
    h.close()


def test_noalloc_limits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300.native import candidates_noalloc
    dev = torch.device("cuda:0")
    z32 = torch.zeros(4, dtype=torch.int32, device=dev)
    g = torch.zeros(4, dtype=torch.int64, device=dev)
    # more nets than the scratch holds
    assert candidates_noalloc(3, (1 << 18) + 1, z32, z32, z32, z32, 2, 0.1, z32, z32, g) == 3
    # a partition entry out of range is rejected before any other kernel runs
    off = torch.tensor([0, 2], dtype=torch.int32, device=dev)
    pins = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    voff = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    inc = torch.tensor([0, 0], dtype=torch.int32, device=dev)
    bad = torch.tensor([0, 5], dtype=torch.int32, device=dev)
    t2 = torch.zeros(2, dtype=torch.int32, device=dev)
    g2 = torch.zeros(2, dtype=torch.int64, device=dev)
    assert candidates_noalloc(2, 1, off, pins, voff, inc, 2, 0.1, bad, t2, g2) == 1
    good = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    assert candidates_noalloc(2, 1, off, pins, voff, inc, 2, 0.5, good, t2, g2, subrounds=1) == 0
    torch.cuda.synchronize()
