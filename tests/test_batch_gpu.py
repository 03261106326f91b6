"""Batched refinement: one launch per phase over many handles, replayed as a CUDA graph.

Each member refined inside a batch must give exactly the result of refining it alone (and the
oracle's), for uneven sizes, mixed k (both record layouts), mixed Phi widths, weights and
sub-round counts, over several calls (graph capture, then replay with continuing rounds).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import build
    build.build()
    oracle.build()


def _members():
    out = []
    specs = [(2, 3000, False, 4, 0), (4, 9000, True, 4, 0), (8, 20000, True, 3, 1), (16, 7000, True, 4, 2),
             (33, 5000, False, 2, 0), (64, 12000, True, 4, 0), (5, 2049, False, 1, 4), (64, 1500, True, 7, 1)]
    for i, (k, n, w, S, pw) in enumerate(specs):
        hg = synth.random_small(4000 + i, n, int(n * 0.9), k, max_size=9, weighted=w, rounds=5)
        out.append((hg, S, pw))
    for hg in synth.config_batch(count=6, n_hi=30_000):
        out.append((hg, 4, 0))
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_alone_and_oracle(graph):
    from paper_2010_10272_gb300 import HGP, Batch
    members = _members()
    hs = [HGP.from_hypergraph(hg, subrounds=S, phi_width=pw, seed=3) for hg, S, pw in members]
    b = Batch(hs, graph=graph)
    got = [b.refine(2), b.refine(3), b.refine(3)]        # capture, new capture (rounds differ), replay
    got = np.concatenate(got, axis=1)
    for i, (hg, S, pw) in enumerate(members):
        o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=3)
        want, _ = o.refine(8)
        np.testing.assert_array_equal(got[i, :, :5], want)
        np.testing.assert_array_equal(hs[i].partition(), o.partition())
        np.testing.assert_array_equal(hs[i].block_weights(), o.block_weights())
        assert hs[i].objective() == o.objective() == hs[i].objective_from_phi()
        assert hs[i].info()["next_round"] == 8
        # a handle refined alone after the batch continues the same sequence
        alone = hs[i].refine(1)[:, :5]
        np.testing.assert_array_equal(alone, o.refine(1)[0])
    assert b.launch_count() > 0
    b.close()


def test_single_handle_graph_mode_replay():
    from paper_2010_10272_gb300 import HGP
    hg = synth.random_small(77, 30000, 28000, 64, max_size=10, weighted=True, rounds=6)
    h = HGP.from_hypergraph(hg, subrounds=4, graph=1)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4)
    for r in (2, 2, 2, 1):                 # capture, replay, replay, re-capture
        np.testing.assert_array_equal(h.refine(r)[:, :5], o.refine(r)[0])
    np.testing.assert_array_equal(h.partition(), o.partition())
    h.set_partition(hg.part)              # reset also restarts the device round state
    o2 = oracle.Oracle.from_hypergraph(hg, subrounds=4)
    np.testing.assert_array_equal(h.refine(2)[:, :5], o2.refine(2)[0])


def test_launch_shapes_do_not_change_results_and_autotune_restores_state():
    from paper_2010_10272_gb300 import HGP, Batch
    from paper_2010_10272_gb300.autotune import tune_batch
    members = _members()[:8]

    def make():
        return [HGP.from_hypergraph(hg, subrounds=S, phi_width=pw, seed=3) for hg, S, pw in members]
    ref_handles = make()
    ref = Batch(ref_handles).refine(3)
    for g, a in [(1, 1), (3, 2), (4, 4)]:
        hs = make()
        got = Batch(hs, gain_ctas_per_sm=g, apply_ctas_per_sm=a).refine(3)
        np.testing.assert_array_equal(got[:, :, :6], ref[:, :, :6])
        for h, r in zip(hs, ref_handles):
            np.testing.assert_array_equal(h.partition(), r.partition())
    hs = make()
    before = [h.export_state() for h in hs]
    best = tune_batch(hs, rounds=2, candidates=[(0, 0), (2, 2)], repeats=1)
    assert (best["gain_ctas_per_sm"], best["apply_ctas_per_sm"]) in best["ms"]
    for h, s in zip(hs, before):
        st = h.export_state()
        np.testing.assert_array_equal(st["partition"], s["partition"])
        assert st["next_round"] == s["next_round"] and st["first_round"] == s["first_round"]
    # refining after tuning equals refining a fresh set
    got = Batch(hs).refine(3)
    np.testing.assert_array_equal(got[:, :, :6], ref[:, :, :6])


def test_full_batch_workload_equals_oracle():
    """All 256 instances of the batch workload (n log-uniform 1e3-2e5, |e| = min(2+Zipf(2.5),
    1000), k in {2,4,8,16}, c(v) in U{1..4}, 5 rounds) in one batch with a tuned launch shape,
    each member element by element against the oracle."""
    import os
    from paper_2010_10272_gb300 import HGP, Batch
    from paper_2010_10272_gb300.autotune import tune_batch
    insts = synth.config_batch()
    assert len(insts) == 256
    hs = [HGP.from_hypergraph(hg, subrounds=4) for hg in insts]
    tuned = tune_batch(hs, rounds=1, candidates=[(0, 0), (4, 4), (2, 4)], repeats=1)
    b = Batch(hs, graph=True, gain_ctas_per_sm=tuned["gain_ctas_per_sm"],
              apply_ctas_per_sm=tuned["apply_ctas_per_sm"])
    got = b.refine(insts[0].rounds)
    threads = max(1, os.cpu_count() or 1)
    moved = 0
    for i, hg in enumerate(insts):
        o = oracle.Oracle.from_hypergraph(hg, subrounds=4, threads=threads)
        want, _ = o.refine(hg.rounds)
        np.testing.assert_array_equal(got[i, :, :5], want, err_msg=f"member {i}")
        np.testing.assert_array_equal(hs[i].partition(), o.partition(), err_msg=f"member {i}")
        np.testing.assert_array_equal(hs[i].block_weights(), o.block_weights())
        assert hs[i].objective() == o.objective() == hs[i].objective_from_phi()
        moved += int(want[:, 2].sum())
        o.close()
    assert moved > 100_000
    b.close()
    for h in hs:
        h.close()


def test_batch_statistics_read_later_and_members_on_other_streams():
    """A batch call queued without statistics, whose statistics are read afterwards
    (hgp_batch_get_stats), equals a call that returns them; members created on their own
    streams are ordered after the batch (read-backs on their streams see its result); a member
    may be destroyed before the batch if the batch is then only destroyed."""
    from paper_2010_10272_gb300 import HGP, Batch, HGPError
    members = _members()[:6]
    streams = [torch.cuda.Stream() for _ in members]
    hs = [HGP.from_hypergraph(hg, subrounds=S, phi_width=pw, seed=3, stream=st)
          for (hg, S, pw), st in zip(members, streams)]
    b = Batch(hs, graph=False, stream=torch.cuda.Stream())
    assert b.refine(3, stats=False) is None
    got = b.stats(3)
    with pytest.raises(HGPError) as ei:
        b.stats(2)                                   # not the last call's round count
    assert ei.value.code == 1
    for i, (hg, S, pw) in enumerate(members):
        o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=3)
        want, _ = o.refine(3)
        np.testing.assert_array_equal(got[i, :, :5], want)
        np.testing.assert_array_equal(hs[i].partition(), o.partition())
    hs[0].close()                                    # before the batch
    b.close()
    np.testing.assert_array_equal(hs[1].refine(1)[:, :5],
                                  oracle.Oracle.from_hypergraph(members[1][0], subrounds=members[1][1], seed=3)
                                  .refine(4)[0][3:])
    for h in hs[1:]:
        h.close()


def test_batches_on_different_streams_share_members():
    """Two batches on two streams over overlapping members, called alternately without reading
    anything in between: each call starts after the other batch's last call on its members, and
    a pipelined reader gets each call's statistics while the next call is already queued."""
    from paper_2010_10272_gb300 import HGP, Batch
    members = _members()[:6]
    hs = [HGP.from_hypergraph(hg, subrounds=S, phi_width=pw, seed=5) for hg, S, pw in members]
    b1 = Batch(hs[:4], graph=False, stream=torch.cuda.Stream())
    b2 = Batch(hs[2:], graph=False, stream=torch.cuda.Stream())
    calls = [(b1, 2), (b2, 1), (b1, 1), (b2, 2), (b1, 2)]
    rounds = [0] * len(hs)
    got = {i: [] for i in range(len(hs))}
    prev = None
    for b, r in calls:
        b.refine(r, stats=False)
        if prev is not None:                         # the previous call, read after this one is queued
            pb, pr = prev
            st = pb.stats(pr)
            for j, h in enumerate(pb.handles):
                got[hs.index(h)].append(st[j, :, :5])
        prev = (b, r)
        for h in b.handles:
            rounds[hs.index(h)] += r
    pb, pr = prev
    st = pb.stats(pr)
    for j, h in enumerate(pb.handles):
        got[hs.index(h)].append(st[j, :, :5])
    for i, (hg, S, pw) in enumerate(members):
        o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=5)
        want, _ = o.refine(rounds[i])
        np.testing.assert_array_equal(np.concatenate(got[i]), want)
        np.testing.assert_array_equal(hs[i].partition(), o.partition())
        assert hs[i].objective() == o.objective()
    b1.close()
    b2.close()
    for h in hs:
        h.close()


def test_batch_partitions_read_back_together():
    """hgp_batch_get_partitions: the listed members' partitions after the last call, back to
    back, in the listed order; equal to each handle's own read-back and to the oracle."""
    from paper_2010_10272_gb300 import HGP, Batch
    members = _members()[:7]
    hs = [HGP.from_hypergraph(hg, subrounds=S, phi_width=pw, seed=6) for hg, S, pw in members]
    b = Batch(hs, graph=False, stream=torch.cuda.Stream())
    b.refine(2, stats=False)
    order = [5, 0, 3, 6]
    parts = b.partitions(order)
    assert b.partitions([]) == []
    for i, p in zip(order, parts):
        o = oracle.Oracle.from_hypergraph(members[i][0], subrounds=members[i][1], seed=6)
        o.refine(2)
        np.testing.assert_array_equal(p, o.partition())
        np.testing.assert_array_equal(p, hs[i].partition())
    b.close()
    for h in hs:
        h.close()


def test_pool_retention_keeps_results():
    """With the library's pool keeping freed memory (hgp_set_pool_retention), handles created
    and destroyed in a loop give the same results as without."""
    from paper_2010_10272_gb300 import HGP
    from paper_2010_10272_gb300.native import set_pool_retention
    hg = synth.random_small(71, 20000, 18000, 8, max_size=9, weighted=True, rounds=3)
    ref = HGP.from_hypergraph(hg, subrounds=4)
    want = ref.refine(3)
    ref.close()
    try:
        set_pool_retention(1 << 30)
        for _ in range(3):
            h = HGP.from_hypergraph(hg, subrounds=4)
            np.testing.assert_array_equal(h.refine(3), want)
            h.close()
    finally:
        set_pool_retention(0)
