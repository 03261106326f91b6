"""Host logic of the serving loop on CPU: admission by a memory budget, waiting while the
queue head does not fit, refusal of a request that can never fit, retirement after its rounds,
latencies from the server clock.  The device handles and the batch are replaced by fakes, so no
GPU is needed; tests/test_serving_gpu.py covers the real thing."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


class FakeHGP:
    live = 0

    def __init__(self, n, m, net_off, pins, k, eps, part, vertex_w=None, net_w=None, **kw):
        self.part = np.asarray(part, np.int32).copy()
        FakeHGP.live += 1

    def partition(self):
        return self.part

    def objective(self):
        return 7

    def close(self):
        FakeHGP.live -= 1


class FakeBatch:
    sizes = []

    def __init__(self, handles, **kw):
        self.handles = handles
        FakeBatch.sizes.append(len(handles))

    def refine(self, rounds, stats=True):
        self.last = rounds
        return np.zeros((len(self.handles), rounds, 7), np.int64) if stats else None

    def stats(self, rounds):
        assert rounds == self.last
        return np.zeros((len(self.handles), rounds, 7), np.int64)

    def done(self):
        return True

    def partitions(self, idx):
        return [self.handles[i].partition() for i in idx]

    def synchronize(self):
        pass

    def close(self):
        pass


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


@pytest.fixture()
def server_cls(monkeypatch):
    from paper_2010_10272_gb300 import serve
    monkeypatch.setattr(serve, "HGP", FakeHGP)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (1 << 40, 1 << 40))
    FakeHGP.live = 0
    FakeBatch.sizes = []
    return serve


def _req(serve, rid, p, rounds):
    hg = synth.serving_request(np.random.SeedSequence(rid), p_lo=p, p_hi=p + 1)
    return serve.Request.from_hypergraph(rid, hg, rounds=rounds)


@pytest.mark.parametrize("depth", [1, 2])
@pytest.mark.parametrize("creators", [0, 3])
def test_admission_by_budget_and_retirement(server_cls, creators, depth):
    serve = server_cls
    reqs = [_req(serve, i, 20_000, 1 + i % 3) for i in range(6)]
    one = reqs[0].footprint()
    srv = serve.Server(memory_budget=int(2.5 * one), reserve_bytes=0, clock=Clock(), creators=creators,
                       depth=depth)
    for r in reqs:
        srv.submit(r)
    done = []
    max_active = 0
    while not srv.idle():
        done.extend(srv.step())
        max_active = max(max_active, len(srv.active))
        assert srv._resident_bytes <= srv.memory_budget
    assert sorted(r.rid for r in done) == list(range(6))
    # at most two requests fit the budget; created on the serving thread, both join one batch
    # (creator threads may finish them one tick apart)
    assert max(FakeBatch.sizes) == 2 if creators == 0 else max(FakeBatch.sizes) <= 2
    assert FakeHGP.live == 0                   # every handle closed on retirement
    for r in done:
        assert r.finished > r.admitted >= r.arrival and r.latency > 0
        np.testing.assert_array_equal(r.result, r.part)
        assert r.stats.shape == (r.rounds, 7)      # one statistics row per round
    srv.close()


def test_request_that_never_fits_is_refused(server_cls):
    serve = server_cls
    small, big = _req(serve, 1, 20_000, 1), _req(serve, 2, 2_000_000, 1)
    srv = serve.Server(memory_budget=int(1.5 * small.footprint()), reserve_bytes=0, clock=Clock())
    srv.submit(big)
    srv.submit(small)
    done = srv.run_until_idle()
    assert [r.rid for r in done] == [1] and [r.rid for r in srv.rejected] == [2]


def test_footprint_grows_with_the_instance(server_cls):
    serve = server_cls
    a = serve.estimate_device_bytes(1000, 1000, 7000, 8, 20, False, False)
    b = serve.estimate_device_bytes(2000, 2000, 14000, 8, 20, False, False)
    c = serve.estimate_device_bytes(3_000_000, 3_000_000, 21_000_000, 8, 20, False, False)
    d = serve.estimate_device_bytes(3_000_000, 3_000_000, 21_000_000, 64, 20, True, True)
    assert a < b < c < d
    # above 2^21 vertices the transpose's pairs (8 bytes per pin) are part of the peak
    assert c >= 21_000_000 * 8


def test_footprint_counts_the_internal_net_order(server_cls):
    """From 2^20 nets with skewed sizes (largest net >= 8x the average) the handle keeps an
    input -> internal net map (4 bytes per net); near-uniform sizes or fewer nets do not."""
    serve = server_cls
    m = 1 << 20
    skewed = serve.estimate_device_bytes(m, m, 7 * m, 8, 200, False, False)     # 1-byte Phi in both
    uniform = serve.estimate_device_bytes(m, m, 7 * m, 8, 50, False, False)
    assert skewed - uniform >= int(m * 4 * 1.05) - 1
    below = serve.estimate_device_bytes(m - 1, m - 1, 7 * (m - 1), 8, 200, False, False)
    below_u = serve.estimate_device_bytes(m - 1, m - 1, 7 * (m - 1), 8, 50, False, False)
    assert below == below_u


class RecordingBatch(FakeBatch):
    """Records the queue of ticks: which requests each tick holds, and how many ticks are
    queued (refined but not yet read) when a new one is queued."""
    queued = []
    log = []

    def refine(self, rounds, stats=True):
        RecordingBatch.log.append((len(RecordingBatch.queued), [h.rid for h in self.handles], rounds))
        RecordingBatch.queued.append(self)
        return super().refine(rounds, stats)

    def done(self):
        return False

    def stats(self, rounds):
        RecordingBatch.queued.remove(self)
        return super().stats(rounds)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipelined_ticks(server_cls, monkeypatch, depth):
    """Ticks are queued up to `depth` deep before the oldest one is read; every request still
    runs exactly its rounds, one tick after another, and retires once."""
    serve = server_cls
    monkeypatch.setattr(serve, "Batch", RecordingBatch)
    RecordingBatch.queued, RecordingBatch.log = [], []
    orig = FakeHGP.__init__

    def init(self, *a, **kw):
        orig(self, *a, **kw)
        self.rid = kw.get("seed")
    monkeypatch.setattr(FakeHGP, "__init__", init)
    want = {0: 2, 1: 3, 2: 5, 3: 5}            # ticks of 2, 1 and 2 rounds
    reqs = [_req(serve, i, 20_000, want[i]) for i in range(4)]
    for i, r in enumerate(reqs):
        r.seed = i
    srv = serve.Server(memory_budget=1 << 40, reserve_bytes=0, clock=Clock(), creators=0, depth=depth)
    for r in reqs:
        srv.submit(r)
    done = srv.run_until_idle()
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    assert max(q for q, _, _ in RecordingBatch.log) == min(depth, 3) - 1   # never more than depth queued
    rounds = {i: 0 for i in range(4)}
    for _, rids, rr in RecordingBatch.log:
        for rid in rids:
            rounds[rid] += rr
    assert rounds == want
    assert [rr for _, _, rr in RecordingBatch.log] == [2, 1, 2]
    for r in done:
        assert r.stats.shape == (want[r.rid], 7)
    assert FakeHGP.live == 0
    srv.close()

