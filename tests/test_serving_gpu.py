"""Serving loop: each request's result is the same alone and in the mix (tolerance 0: the
arithmetic is integer), with requests arriving while others are on the GPU, admission by a
memory budget that forces queueing, and uneven sizes / k / round counts."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import build
    build.build()


def _requests():
    from paper_2010_10272_gb300.serve import Request
    reqs = []
    for i in range(14):
        hg = synth.serving_request(np.random.SeedSequence(500 + i), p_lo=10_000, p_hi=400_000)
        reqs.append(Request.from_hypergraph(i, hg, rounds=1 + i % 4, subrounds=1 + i % 4, seed=i))
    return reqs


def _alone(req):
    from paper_2010_10272_gb300 import HGP
    h = HGP(req.n, req.m, req.net_off, req.pins, req.k, req.eps, req.part, req.vertex_w, req.net_w,
            subrounds=req.subrounds, seed=req.seed)
    st = h.refine(req.rounds)
    out = (h.partition(), h.objective(), st[:, :5].copy())
    h.close()
    return out


@pytest.mark.parametrize("budget,depth,own_streams,tick_streams",
                         [(None, 2, False, 1), (96 << 20, 2, False, 1), (None, 1, False, 1),
                          (96 << 20, 3, False, 1), (None, 2, True, 1), (None, 2, False, 2),
                          (96 << 20, 3, False, 3)])
def test_mix_equals_alone(budget, depth, own_streams, tick_streams):
    """own_streams: no server stream, so every tick's batch runs on a stream of its own;
    tick_streams: ticks take server streams in turn.  Either way the requests that continue
    from one tick to the next are ordered across batches on different streams."""
    from paper_2010_10272_gb300.serve import Server
    reqs = _requests()
    s = None if own_streams else torch.cuda.Stream()
    srv = Server(stream=s, memory_budget=budget, reserve_bytes=0, depth=depth, tick_streams=tick_streams)
    done = []
    pending = list(reqs)
    # arrivals in waves while earlier requests are still running
    while pending or not srv.idle():
        for _ in range(3):
            if pending:
                srv.submit(pending.pop(0))
        done.extend(srv.step())
    srv.close()
    assert sorted(r.rid for r in done) == list(range(len(reqs)))
    if budget is not None:
        assert srv.ticks > max(r.rounds for r in reqs) + 2   # the budget forced queueing
    for r in done:
        part, obj, objs = _alone(r)
        np.testing.assert_array_equal(r.result, part)
        assert r.objective == obj
        np.testing.assert_array_equal(r.stats[:, :5], objs)
        assert r.finished >= r.admitted >= r.arrival


def test_footprint_estimate_covers_creation():
    from paper_2010_10272_gb300 import HGP
    from paper_2010_10272_gb300.serve import Request
    hg = synth.serving_request(np.random.SeedSequence(9), p_lo=2_000_000, p_hi=2_000_001)
    req = Request.from_hypergraph(0, hg)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    h = HGP.from_hypergraph(hg)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    print("device bytes used by one request:", used, "estimate:", req.footprint())
    assert used <= req.footprint()
    h.close()


def test_request_sizes_against_oracle():
    """One serving request per size decade up to the workload's largest (10^4 .. 5*10^6 pins),
    served together in the mix, each element by element against the oracle as well as against
    the same request refined alone."""
    import os
    import oracle
    from paper_2010_10272_gb300.serve import Request, Server
    oracle.build()
    sizes = [10_000, 100_000, 1_000_000, 5_000_000]
    reqs = []
    for i, p in enumerate(sizes):
        hg = synth.serving_request(np.random.SeedSequence(700 + i), p_lo=p, p_hi=p + 1)
        reqs.append(Request.from_hypergraph(i, hg, seed=i))
    assert reqs[-1].num_pins > 4_000_000
    srv = Server(stream=torch.cuda.Stream(), reserve_bytes=0)
    for r in reqs:
        srv.submit(r)
    done = srv.run_until_idle()
    srv.close()
    assert sorted(r.rid for r in done) == list(range(len(sizes)))
    threads = max(1, os.cpu_count() or 1)
    for r in done:
        o = oracle.Oracle(r.n, r.m, r.net_off, r.pins, r.k, r.eps, r.part, r.vertex_w, r.net_w,
                          r.subrounds, r.seed, threads=threads)
        want, _ = o.refine(r.rounds)
        np.testing.assert_array_equal(r.stats[:, :5], want, err_msg=f"request {r.rid}")
        np.testing.assert_array_equal(r.result, o.partition())
        assert r.objective == o.objective()
        part, obj, st = _alone(r)
        np.testing.assert_array_equal(part, r.result)
        assert obj == r.objective


def test_concurrent_creation_from_threads():
    """Handles created at the same time from several host threads (each on its own stream, as
    the server's creator threads do), with k and Phi widths differing from thread to thread,
    equal handles created one after another."""
    import concurrent.futures
    import threading
    from paper_2010_10272_gb300 import HGP
    specs = [(2 + (i % 5) * 7, 3000 + 500 * (i % 7)) for i in range(48)]
    hgs = [synth.random_small(880 + i, n, n, k, max_size=7 + (i % 3) * 150, weighted=i % 2 == 0, rounds=2)
           for i, (k, n) in enumerate(specs)]
    tls = threading.local()
    dev = torch.cuda.current_device()

    def make(hg):
        s = getattr(tls, "s", None)
        if s is None:
            torch.cuda.set_device(dev)
            s = tls.s = torch.cuda.Stream()
        h = HGP.from_hypergraph(hg, stream=s)
        st = h.refine(2)
        out = (h.partition(), st[:, :5].copy(), h.info()["phi_width"])
        h.close()
        return out

    for _ in range(2):
        with concurrent.futures.ThreadPoolExecutor(8) as ex:
            got = list(ex.map(make, hgs))
        for hg, (part, st, w) in zip(hgs, got):
            h = HGP.from_hypergraph(hg)
            np.testing.assert_array_equal(h.refine(2)[:, :5], st)
            np.testing.assert_array_equal(h.partition(), part)
            assert h.info()["phi_width"] == w
            h.close()
    assert len({w for _, _, w in got}) == 2          # both entry widths were created concurrently
