"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Every quantity is integer, so the bar is bit-exact: partition, Phi table, Lambda bitsets,
block weights, objective and per-round (objective, candidates, approved, eligible, max
block weight).  Sizes span several 2048-vertex tiles with ragged tails.
"""
import numpy as np
import pytest

import oracle
import synth
from golden_io import load_all
from paper_2010_10272_gb300 import HGP
from parity_util import compare_state, run_both

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = load_all()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import build as b
    b.build()
    import oracle as o
    o.build()




# ---------------------------------------------------------------- hand-derived fixtures
@pytest.mark.parametrize("g", GOLDEN, ids=[g.name for g in GOLDEN])
def test_golden(g):
    h = HGP(g.n, g.m, g.net_off, g.pins, g.k, g.eps, g.part, g.vertex_w, g.net_w,
            subrounds=g.subrounds, seed=g.seed)
    assert h.info()["lmax"] == g.lmax
    assert h.objective() == g.objective
    stats = h.refine(len(g.rounds))[:, :5]
    assert [tuple(r) for r in stats.tolist()] == list(g.rounds)
    np.testing.assert_array_equal(h.partition(), g.final)


# ---------------------------------------------------------------- seeded random instances
CASES = [
    # (seed, n, m, k, max_size, weighted, S, phi_width)
    (1, 5000, 4000, 2, 6, False, 4, 0),
    (2, 7001, 6000, 3, 8, True, 1, 0),
    (3, 6143, 9000, 8, 12, False, 4, 0),
    (4, 9999, 8000, 16, 10, True, 7, 2),
    (5, 4097, 5000, 31, 9, False, 2, 4),
    (6, 4500, 5000, 32, 9, True, 3, 0),
    (7, 6000, 5500, 33, 9, False, 4, 1),
    (8, 8191, 7000, 64, 12, True, 5, 0),
    (9, 3000, 2000, 64, 40, False, 64, 2),
    (10, 2049, 2500, 5, 300, True, 4, 1),    # nets > 255 pins -> wide tier with 1-byte Phi
]


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-n{c[1]}-k{c[3]}-S{c[6]}-w{c[7]}" for c in CASES])
def test_random_instances(case):
    seed, n, m, k, max_size, weighted, S, w = case
    hg = synth.random_small(seed, n, m, k, max_size=max_size, weighted=weighted, rounds=4)
    h, o, _ = run_both(hg, rounds=4, S=S, seed=seed, phi_width=w)
    if case[0] == 10:
        assert h.info()["wide_nets"] > 0


def test_small_config_full_size():
    hg = synth.config_small()
    run_both(hg, S=4)


def test_batch_members():
    for hg in synth.config_batch(count=6, n_hi=20_000):
        run_both(hg, S=4)


def test_powerlaw_scaled_with_wide_tier():
    hg = synth.config_powerlaw(scale=0.002)          # n = m = 100k, k = 64, weighted nets
    h, o, _ = run_both(hg, S=4, phi_width=1, check_phi=False)
    assert h.info()["wide_nets"] > 0


def test_powerlaw_scaled_u16():
    hg = synth.config_powerlaw(scale=0.004)
    h, _, stats = run_both(hg, S=4, phi_width=2, check_phi=False)
    assert h.info()["phi_width"] == 2
    assert stats[0, 2] > 0


def test_phi_width_choices():
    # automatic: chosen by the largest net (2 bytes here); forced 1 byte: the nets above 255
    # pins go to the wide table; both give the oracle's rounds
    hg = synth.config_powerlaw(scale=0.004)
    h, _, _ = run_both(hg, S=4, check_phi=False)
    assert h.info()["phi_width"] == 2
    h1, _, _ = run_both(hg, S=4, phi_width=1, check_phi=False)
    assert h1.info()["phi_width"] == 1 and h1.info()["wide_nets"] > h.info()["wide_nets"]


# ---------------------------------------------------------------- approval edge cases
def test_saturated_blocks_and_large_gains():
    """Net weights up to 2^20 push gains past the 4094 exact histogram bins, so the
    threshold is resolved digit by digit; a tight eps saturates every block."""
    rng = np.random.default_rng(11)
    hg = synth.random_small(11, 6000, 7000, 4, max_size=5, weighted=False, eps=0.01, rounds=5)
    hg.net_w = rng.integers(1, 1 << 20, size=hg.m, dtype=np.int32)
    hg.vertex_w = rng.integers(1, 3, size=hg.n, dtype=np.int32)
    run_both(hg, S=2)


def test_ties_everywhere_unit_weights():
    # many equal gains and unit weights: ties at the threshold span many tiles
    hg = synth.planted(3, 60_000, 60_000, 2, synth.poisson_sizes(2.0), 0.9, 0.45, eps=0.001, rounds=3)
    run_both(hg, S=1)


def test_unbalanced_start():
    hg = synth.random_small(12, 5000, 5000, 6, max_size=6, weighted=True, eps=0.03, rounds=5)
    part = hg.part.copy()
    part[: hg.n // 2] = 0
    run_both(hg, S=3, part=part)


# ---------------------------------------------------------------- degenerate inputs
def test_degenerate_nets_and_vertices():
    # empty nets, single-pin nets, isolated vertices, a hub vertex in every other net
    rng = np.random.default_rng(5)
    n, m, k = 3000, 4000, 4
    nets = []
    for e in range(m):
        r = e % 5
        if r == 0:
            nets.append([])
        elif r == 1:
            nets.append([int(rng.integers(0, n))])
        else:
            s = set(rng.choice(n - 100, size=int(rng.integers(2, 8)), replace=False).tolist())
            if e % 2 == 0:
                s.add(n - 1)          # hub
            nets.append(sorted(s))
    off = np.zeros(m + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(x) for x in nets])
    pins = np.array([v for x in nets for v in x], dtype=np.int32)
    part = rng.integers(0, k, size=n).astype(np.int32)
    hg = synth.Hypergraph("degenerate", n, m, k, 0.05, off, pins, part, None, None, 4)
    run_both(hg, S=2)


def test_no_nets_and_single_vertex():
    for n, m in ((1, 0), (5, 0), (1, 3)):
        off = np.zeros(m + 1, dtype=np.int64)
        if m == 3:
            off[:] = [0, 0, 1, 1]
        pins = np.zeros(int(off[-1]), dtype=np.int32)
        hg = synth.Hypergraph("tiny", n, m, 2, 0.5, off, pins, np.zeros(n, np.int32), None, None, 2)
        run_both(hg, S=1)


def test_all_vertices_in_one_block_k64():
    hg = synth.random_small(13, 3000, 3000, 64, max_size=6, rounds=3)
    run_both(hg, S=4, part=np.zeros(hg.n, np.int32))


# ---------------------------------------------------------------- gain step alone
@pytest.mark.parametrize("k,S,weighted", [(2, 4, False), (8, 3, True), (64, 2, True), (33, 1, False)])
def test_candidates_match_oracle(k, S, weighted):
    hg = synth.random_small(20 + k, 9000, 8000, k, max_size=10, weighted=weighted)
    h = HGP.from_hypergraph(hg, subrounds=S, seed=3)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=3)
    for step in range(2):
        for s in range(S):
            t_h, g_h = h.debug_candidates(s)
            t_o, g_o = o.candidates(s)
            np.testing.assert_array_equal(t_h, t_o)
            np.testing.assert_array_equal(g_h, g_o)
        h.refine(1)
        o.refine(1)


# ---------------------------------------------------------------- API semantics
def test_refine_split_equals_whole():
    hg = synth.random_small(30, 8000, 8000, 8, max_size=8, weighted=True, rounds=6)
    run_both(hg, rounds=6, S=4, chunks=[1, 2, 3])
    run_both(hg, rounds=6, S=4, chunks=[6])


def test_repeat_runs_identical():
    hg = synth.random_small(31, 10000, 9000, 16, max_size=8, weighted=True, rounds=4)
    res = []
    for _ in range(3):
        h = HGP.from_hypergraph(hg, subrounds=4, seed=9)
        st = h.refine(4)
        res.append((st, h.partition(), h.phi()))
    for st, p, phi in res[1:]:
        np.testing.assert_array_equal(st, res[0][0])
        np.testing.assert_array_equal(p, res[0][1])
        np.testing.assert_array_equal(phi, res[0][2])


def test_set_partition_equals_fresh_create():
    hg = synth.random_small(32, 6000, 6000, 4, max_size=7, rounds=3)
    h = HGP.from_hypergraph(hg, subrounds=4)
    h.refine(3)
    h.set_partition(hg.part)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4)
    compare_state(h, o)
    np.testing.assert_array_equal(h.refine(3)[:, :5], o.refine(3)[0])
    compare_state(h, o)


def test_device_inputs_and_stream():
    hg = synth.random_small(33, 5000, 5000, 8, max_size=7, weighted=True, rounds=3)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    s = torch.cuda.Stream()
    h = HGP(hg.n, hg.m, t(hg.net_off), t(hg.pins), hg.k, hg.eps, t(hg.part), t(hg.vertex_w),
            t(hg.net_w), subrounds=4, device=True, stream=s)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4)
    np.testing.assert_array_equal(h.refine(3)[:, :5], o.refine(3)[0])
    out = torch.empty(hg.n, dtype=torch.int32, device=dev)
    h.partition(out_device=out)
    np.testing.assert_array_equal(out.cpu().numpy(), o.partition())


def test_check_mode():
    hg = synth.random_small(34, 4000, 4000, 5, max_size=7, weighted=True, rounds=3)
    h = HGP.from_hypergraph(hg, subrounds=2, debug=1)
    h.refine(3)


def test_check_mode_reports_an_injected_fault():
    """Fault injection on the host (debug bit 4: the maintained objective loses one unit after
    each refine, as a dropped update would): check mode returns HGP_ERR_INTERNAL, the handle
    still answers (the maintained value is the recomputed one minus one, the partition is the
    oracle's), a new partition rebuilds the state, and destroying the handle gives back every
    byte it took on the device (measured on a second identical cycle, after the first one has
    loaded every kernel it uses)."""
    import torch
    from paper_2010_10272_gb300 import HGPError
    hg = synth.random_small(35, 5000, 4500, 6, max_size=7, weighted=True, rounds=2)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=3)
    o.refine(2)

    def cycle():
        h = HGP.from_hypergraph(hg, subrounds=3, debug=1 | 16)
        with pytest.raises(HGPError) as ei:
            h.refine(2)
        assert ei.value.code == 6
        np.testing.assert_array_equal(h.partition(), o.partition())
        assert h.objective_from_phi() == o.objective() == h.objective() + 1
        h.set_partition(hg.part)
        assert h.objective() == h.objective_from_phi()
        # without check mode the injected loss goes unnoticed by refine itself
        h2 = HGP.from_hypergraph(hg, subrounds=3, debug=16)
        h2.refine(1)
        assert h2.objective() == h2.objective_from_phi() - 1
        h.close()
        h2.close()
        torch.cuda.synchronize()

    cycle()
    free0, _ = torch.cuda.mem_get_info()
    cycle()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0


# ---------------------------------------------------------------- error codes
def _err(fn):
    from paper_2010_10272_gb300 import HGPError
    with pytest.raises(HGPError) as ei:
        fn()
    return ei.value.code


def test_error_codes():
    off = np.array([0, 2, 3], dtype=np.int64)
    pins = np.array([0, 1, 2], dtype=np.int32)
    part = np.array([0, 1, 0], dtype=np.int32)
    ok = dict(n=3, m=2, net_off=off, pins=pins, k=2, eps=0.1, part=part)

    def mk(**kw):
        a = dict(ok)
        a.update(kw)
        return lambda: HGP(a["n"], a["m"], a["net_off"], a["pins"], a["k"], a["eps"], a["part"],
                           a.get("vertex_w"), a.get("net_w"), subrounds=a.get("subrounds", 4))
    HGP(3, 2, off, pins, 2, 0.1, part).close()
    assert _err(mk(k=1)) == 1
    assert _err(mk(k=65)) == 3
    assert _err(mk(eps=0.0)) == 1
    assert _err(mk(eps=1.0)) == 1
    assert _err(mk(part=np.array([0, 2, 0], np.int32))) == 1
    assert _err(mk(pins=np.array([0, 5, 2], np.int32))) == 1                   # out of range
    assert _err(mk(pins=np.array([1, 0, 2], np.int32))) == 1                   # not increasing
    assert _err(mk(pins=np.array([1, 1, 2], np.int32))) == 1                   # duplicate
    assert _err(mk(net_off=np.array([0, 3, 2], np.int64))) == 1                # decreasing
    assert _err(mk(net_off=np.array([1, 2, 3], np.int64))) == 1                # not from 0
    assert _err(mk(vertex_w=np.array([1, 0, 1], np.int32))) == 1
    assert _err(mk(net_w=np.array([1, -3], np.int32))) == 1
    assert _err(mk(subrounds=65)) == 3
    # vertex 1 lies in both nets; their weights sum to 2^31 -> unsupported
    assert _err(mk(net_w=np.array([1 << 30, 1 << 30], np.int32),
                   pins=np.array([0, 1, 1, 2], np.int32),
                   net_off=np.array([0, 2, 4], np.int64))) == 3


@pytest.mark.parametrize("debug,device", [(0, True), (2, False), (4, False), (2 | 4, True)],
                         ids=["device", "bucketed", "reordered", "bucketed-reordered-device"])
def test_invalid_inputs_every_creation_path(debug, device):
    """Host inputs of small instances are checked while the creation is already queued (the
    kernels after the checks skip flagged input; the verdict comes with the final read-back);
    device inputs wait for the checks first.  Both reject the same inputs, whatever the
    transpose and net order, including pins far outside [0, n) that the bucketed transpose would
    otherwise use as bucket indices."""
    import torch
    from paper_2010_10272_gb300 import HGP
    rng = np.random.default_rng(8)
    n, m = 5000, 4000
    sizes = rng.integers(1, 7, size=m)
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    pins = np.concatenate([np.sort(rng.choice(n, size=int(s), replace=False)) for s in sizes]).astype(np.int32)
    part = rng.integers(0, 4, size=n).astype(np.int32)
    vw = rng.integers(1, 4, size=n).astype(np.int32)
    nw = rng.integers(1, 4, size=m).astype(np.int32)

    def make(pins_=pins, part_=part, vw_=vw, nw_=nw):
        if device:
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            return HGP(n, m, t(off), t(pins_), 4, 0.05, t(part_), t(vw_), t(nw_), debug=debug, device=True)
        return HGP(n, m, off, pins_, 4, 0.05, part_, vw_, nw_, debug=debug)

    h = make()
    o = oracle.Oracle(n, m, off, pins, 4, 0.05, part, vw, nw, 4, 0)
    compare_state(h, o)
    h.close()
    far = pins.copy()
    far[len(far) // 2] = (1 << 30) + 7
    neg = pins.copy()
    neg[3] = -(1 << 29)
    bad_part = part.copy()
    bad_part[17] = 200
    bad_vw = vw.copy()
    bad_vw[5] = 0
    bad_nw = nw.copy()
    bad_nw[9] = -1
    assert _err(lambda: make(pins_=far)) == 1
    assert _err(lambda: make(pins_=neg)) == 1
    assert _err(lambda: make(part_=bad_part)) == 1
    assert _err(lambda: make(vw_=bad_vw)) == 1
    assert _err(lambda: make(nw_=bad_nw)) == 1
    h = make()                                     # the device is fine afterwards
    compare_state(h, o)
    h.close()


def test_moved_pins_and_profile():
    """moved_pins = sum of degrees of the vertices the oracle moved; profiling accounts for
    every kernel the rounds launch."""
    hg = synth.random_small(35, 20000, 18000, 8, max_size=9, weighted=True, rounds=3)
    h = HGP.from_hypergraph(hg, subrounds=4)
    h.set_profiling(True)
    l0 = h.launch_count()
    st = h.refine(3)
    launched = h.launch_count() - l0
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4)
    _, moves = o.refine(3, log_moves=True)
    deg = np.bincount(hg.pins, minlength=hg.n)
    for r in range(3):
        sel = moves[(moves[:, 0] // 4) == r]
        assert st[r, 5] == deg[sel[:, 1]].sum()
    prof = h.profile()
    assert sum(v[1] for v in prof.values()) == launched
    assert prof["gain"][1] == 3 * 4 and prof["apply"][1] == 3 * 4
    assert all(v[0] > 0 for name, v in prof.items() if name != "revert")
    assert prof["revert"] == (0.0, 0)                 # revert variant off


@pytest.mark.parametrize("k,graph", [(8, 0), (8, 1), (64, 0), (64, 1)])
def test_checkpoint_resume(k, graph):
    """refine(2); export; import into a fresh handle; refine(3) == refine(5) (and the oracle)."""
    hg = synth.random_small(36 + k, 15000, 14000, k, max_size=9, weighted=True, rounds=5)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=3, seed=4)
    want, _ = o.refine(5)
    a = HGP.from_hypergraph(hg, subrounds=3, seed=4, graph=graph)
    first = a.refine(2)[:, :5]
    st = a.export_state()
    assert st["next_round"] == 2 and st["first_round"] == 0
    b = HGP.from_hypergraph(hg, subrounds=3, seed=4, graph=graph)
    b.import_state(st)
    rest = b.refine(3)[:, :5]
    np.testing.assert_array_equal(np.concatenate([first, rest]), want)
    np.testing.assert_array_equal(b.partition(), o.partition())
    assert b.objective() == o.objective()
    # a state exported before any round resumes as a fresh handle
    c = HGP.from_hypergraph(hg, subrounds=3, seed=4)
    s0 = c.export_state()
    assert s0["first_round"] == 1 and not s0["moved_nets"].any()
    d = HGP.from_hypergraph(hg, subrounds=3, seed=4)
    d.import_state(s0)
    np.testing.assert_array_equal(d.refine(5)[:, :5], want)


@pytest.mark.parametrize("k,weighted,frac", [(2, False, 0.3), (8, True, 0.5), (64, True, 0.2), (40, False, 1.0)])
def test_exact_gains_match_oracle(k, weighted, frac):
    """Lemma 1 on the GPU against the oracle's sequential replay, random move sequences."""
    rng = np.random.default_rng(k)
    hg = synth.random_small(70 + k, 20000, 18000, k, max_size=12, weighted=weighted)
    h = HGP.from_hypergraph(hg)
    o = oracle.Oracle.from_hypergraph(hg)
    verts = rng.permutation(hg.n)[: int(frac * hg.n)]
    to = rng.integers(0, k - 1, size=verts.size)
    a = hg.part[verts]
    to = np.where(to >= a, to + 1, to)
    moves = np.stack([verts, a, to], axis=1).astype(np.int32)
    np.testing.assert_array_equal(h.exact_gains(moves), o.exact_gains(moves))
    np.testing.assert_array_equal(h.partition(), hg.part)      # state unchanged
    from paper_2010_10272_gb300 import HGPError
    bad = moves[:2].copy()
    bad[1, 0] = bad[0, 0]                                        # vertex twice
    with pytest.raises(HGPError):
        h.exact_gains(bad)


def test_exact_gains_of_lp_moves_sum_to_objective_change():
    hg = synth.random_small(99, 30000, 30000, 16, max_size=8, weighted=True, rounds=1)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=1)
    _, log = o.refine(1, log_moves=True)
    h = HGP.from_hypergraph(hg, subrounds=1)
    g = h.exact_gains(log[:, 1:].astype(np.int32))
    st = h.refine(1)
    o0 = oracle.Oracle.from_hypergraph(hg, subrounds=1)
    assert o0.objective() - st[0, 0] == g.sum()


# ---------------------------------------------------------------- creation paths
@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[7], CASES[9]],
                         ids=["k2", "k16-w2", "k64", "wide"])
def test_bucketed_transpose_forced(case):
    """The bucketed net -> vertex transpose (used above 2^21 vertices) forced at small sizes
    (down to 256-vertex buckets): same rounds, Phi and partition as the oracle."""
    seed, n, m, k, max_size, weighted, S, w = case
    hg = synth.random_small(seed, n, m, k, max_size=max_size, weighted=weighted, rounds=4)
    h = HGP.from_hypergraph(hg, subrounds=S, seed=seed, phi_width=w, debug=2)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=seed)
    compare_state(h, o)
    np.testing.assert_array_equal(h.refine(4)[:, :5], o.refine(4)[0])
    compare_state(h, o)


def test_bucketed_transpose_degenerate():
    # empty nets, single-pin nets, isolated vertices, a vertex in every net
    n, m = 3000, 2000
    rng = np.random.default_rng(5)
    nets = []
    for e in range(m):
        s = int(rng.integers(0, 6))
        pins = set(rng.choice(n - 100, size=s, replace=False).tolist()) if s else set()
        if e % 3 == 0:
            pins.add(n - 101)                        # the hub
        nets.append(sorted(pins))
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in nets])
    pins = np.array([v for x in nets for v in x], np.int32)
    part = rng.integers(0, 4, size=n).astype(np.int32)
    h = HGP(n, m, off, pins, 4, 0.1, part, subrounds=2, debug=2)
    o = oracle.Oracle(n, m, off, pins, 4, 0.1, part, None, None, 2, 0)
    compare_state(h, o)
    np.testing.assert_array_equal(h.refine(3)[:, :5], o.refine(3)[0])
    compare_state(h, o)


def test_launch_shape_and_instance_autotune():
    """Launch shapes never change results; the instance tuner returns one of its candidates,
    and a handle created with the tuned choices matches the oracle."""
    from paper_2010_10272_gb300.autotune import tune_instance
    hg = synth.random_small(91, 20000, 18000, 16, max_size=300, weighted=True, rounds=3)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4, seed=1)
    want, _ = o.refine(3)
    for g, a in [(1, 1), (2, 3), (4, 4)]:
        h = HGP.from_hypergraph(hg, subrounds=4, seed=1, gain_ctas_per_sm=g, apply_ctas_per_sm=a)
        np.testing.assert_array_equal(h.refine(3)[:, :5], want)
    h = HGP.from_hypergraph(hg, subrounds=4, seed=1)
    h.refine(1)
    h.set_launch_shape(3, 1)
    np.testing.assert_array_equal(h.refine(2)[:, :5], want[1:])
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    best = tune_instance(hg.n, hg.m, dev(hg.net_off), dev(hg.pins), hg.k, hg.eps, dev(hg.part),
                         dev(hg.vertex_w), dev(hg.net_w), rounds=2, shapes=[(0, 0), (2, 2)], repeats=1,
                         seed=1)
    assert best["phi_width"] in (1, 2) and (best["gain_ctas_per_sm"], best["apply_ctas_per_sm"]) in [(0, 0), (2, 2)]
    ht = HGP.from_hypergraph(hg, subrounds=4, seed=1, phi_width=best["phi_width"],
                             gain_ctas_per_sm=best["gain_ctas_per_sm"], apply_ctas_per_sm=best["apply_ctas_per_sm"])
    np.testing.assert_array_equal(ht.refine(3)[:, :5], want)
