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

import oracle
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
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=7)
    for s in (0, 1):                       # two calls in a row share the scratch array
        rc = candidates_noalloc(hg.n, hg.m, *args, hg.k, hg.eps, t(hg.part), target, gain,
                                vertex_w=t(hg.vertex_w), net_w=t(hg.net_w), subrounds=S, seed=7, s=s)
        assert rc == 0
        torch.cuda.synchronize()
        want_t, want_g = h.debug_candidates(s)
        np.testing.assert_array_equal(target.cpu().numpy(), want_t)
        np.testing.assert_array_equal(gain.cpu().numpy(), want_g)
        # and directly against the oracle's candidates of the same sub-round
        o_t, o_g = o.candidates(s)
        np.testing.assert_array_equal(target.cpu().numpy(), o_t)
        np.testing.assert_array_equal(gain.cpu().numpy(), o_g)
        assert (want_t >= 0).any()
    h.close()
    o.close()


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


def _tiny(dev):
    """nets {0,1}, {1,2}, {0,2,3}; 4 vertices; a consistent transpose."""
    i32 = lambda a: torch.tensor(a, dtype=torch.int32, device=dev)  # noqa: E731
    return dict(off=i32([0, 2, 4, 7]), pins=i32([0, 1, 1, 2, 0, 2, 3]),
                voff=i32([0, 2, 4, 6, 7]), inc=i32([0, 2, 0, 1, 1, 2, 2]),
                part=i32([0, 1, 0, 1]), vw=i32([1, 1, 1, 1]), nw=i32([1, 2, 3]))


def _call(a, **over):
    from paper_2010_10272_gb300.native import candidates_noalloc
    a = dict(a, **over)
    dev = a["off"].device
    t = torch.empty(4, dtype=torch.int32, device=dev)
    g = torch.empty(4, dtype=torch.int64, device=dev)
    rc = candidates_noalloc(4, a["off"].numel() - 1, a["off"], a["pins"], a["voff"], a["inc"], 2, 0.5,
                            a["part"], t, g, vertex_w=a["vw"], net_w=a["nw"], subrounds=1)
    torch.cuda.synchronize()
    return rc, t, g


def test_noalloc_rejects_each_invalid_input():
    """Every validation rule returns HGP_ERR_INVALID (1), and a valid call still works after
    the rejected ones (the error flag is cleared on every call)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    a = _tiny(dev)
    i32 = lambda x: torch.tensor(x, dtype=torch.int32, device=dev)  # noqa: E731
    assert _call(a)[0] == 0
    bad_cases = {
        "net offsets not monotone": dict(off=i32([0, 4, 2, 7])),
        "net offsets end before P": dict(off=i32([0, 2, 4, 6]), pins=i32([0, 1, 1, 2, 0, 2, 3])),
        "vertex offsets not monotone": dict(voff=i32([0, 3, 2, 6, 7])),
        "vertex offsets end != P": dict(voff=i32([0, 2, 4, 6, 6])),
        "pin out of range": dict(pins=i32([0, 1, 1, 2, 0, 2, 4])),
        "incident net out of range": dict(inc=i32([0, 2, 0, 1, 1, 2, 3])),
        "pin repeated in a net": dict(pins=i32([0, 0, 1, 2, 0, 2, 3])),
        "pins not increasing": dict(pins=i32([1, 0, 1, 2, 0, 2, 3])),
        "nets of a vertex not increasing": dict(inc=i32([2, 0, 0, 1, 1, 2, 2])),
        "not the transpose": dict(inc=i32([0, 2, 0, 1, 1, 2, 1])),
        "vertex weight 0": dict(vw=i32([1, 0, 1, 1])),
        "net weight negative": dict(nw=i32([1, -2, 3])),
        "partition entry out of range": dict(part=i32([0, 1, 2, 1])),
    }
    for name, over in bad_cases.items():
        assert _call(a, **over)[0] == 1, name
    rc, t, g = _call(a)
    assert rc == 0


def test_noalloc_without_nets():
    """m = 0: no records are written; every vertex has W = 0 and no candidate."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300.native import candidates_noalloc
    dev = torch.device("cuda:0")
    n = 1000
    off = torch.zeros(1, dtype=torch.int32, device=dev)
    voff = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    empty = torch.zeros(0, dtype=torch.int32, device=dev)
    part = torch.arange(n, dtype=torch.int32, device=dev) % 3
    t = torch.full((n,), 7, dtype=torch.int32, device=dev)
    g = torch.full((n,), 7, dtype=torch.int64, device=dev)
    for s in (0, 1):
        rc = candidates_noalloc(n, 0, off, empty, voff, empty, 3, 0.1, part, t, g, subrounds=2, s=s)
        assert rc == 0
        torch.cuda.synchronize()
        assert bool((t == -1).all()) and bool((g == 0).all())


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")   # the refused call captures nothing
def test_noalloc_refuses_stream_capture():
    """The call reads its validation result back to the host, which a capture forbids: it
    returns HGP_ERR_INVALID instead of invalidating the capture."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    a = _tiny(dev)
    assert _call(a)[0] == 0                    # first call on the device: set-up outside capture
    from paper_2010_10272_gb300.native import candidates_noalloc
    t = torch.empty(4, dtype=torch.int32, device=dev)
    g = torch.empty(4, dtype=torch.int64, device=dev)
    s = torch.cuda.Stream(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        graph.capture_begin()
        rc = candidates_noalloc(4, 3, a["off"], a["pins"], a["voff"], a["inc"], 2, 0.5, a["part"], t, g,
                                vertex_w=a["vw"], net_w=a["nw"], subrounds=1, stream=s)
        graph.capture_end()
    assert rc == 1
    assert _call(a)[0] == 0
