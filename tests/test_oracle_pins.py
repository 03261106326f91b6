"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

No expected value here comes from the oracle itself or from the CUDA library:
* hand-derived fixtures (tests/golden/, derivations in each file);
* the published SplitMix64 test vector;
* L_max closed forms;
* brute force on tiny inputs (objective from connectivity sets, gains as objective
  differences, eligibility from neighbourhoods), see tests/brute.py;
* invariants (sum of Phi over blocks = |e|, block weights sum to c(V), balance);
* exhaustive optimal bipartitions of hypergraphs with at most 12 vertices.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from brute import Tiny, lp_rounds, random_tiny, subround
from golden_io import load_all

GOLDEN = load_all()


def make_oracle(t: Tiny, part, S=4, seed=0):
    off, pins = t.csr()
    vw = None if all(x == 1 for x in t.vw) else np.array(t.vw, dtype=np.int32)
    nw = None if all(x == 1 for x in t.nw) else np.array(t.nw, dtype=np.int32)
    return oracle.Oracle(t.n, t.m, off, pins, t.k, t.eps, np.array(part, dtype=np.int32),
                         vw, nw, S, seed)


# --- published values and closed forms -------------------------------------------------

def test_splitmix64_published_vector():
    # SplitMix64 with seed 0 emits mix(1*gamma), mix(2*gamma), mix(3*gamma) =
    # 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f (Steele, Lea, Flood 2014)
    gamma = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for i, want in enumerate(expect, 1):
        assert oracle.mix64((i * gamma) & ((1 << 64) - 1)) == want


def test_subround_hash_matches_definition():
    for seed in (0, 1, 0xDEADBEEF12345678):
        for r in (0, 1, 7, 123456):
            for u in (0, 1, 2, 31, 1 << 20, (1 << 31) - 1):
                for S in (1, 2, 3, 4, 7):
                    assert oracle.subround_of(seed, r, u, S) == subround(seed, r, u, S)


@pytest.mark.parametrize("total,k,eps,want", [
    (10_000, 2, 0.03, 5150),          # ceil(5000) * 1.03
    (2_000_000, 8, 0.03, 257_500),    # 250000 * 1.03
    (50_000_000, 64, 0.03, 804_687),  # 781250 * 1.03 = 804687.5 -> floor
    (7, 2, 0.03, 4),                  # ceil(3.5) = 4; 4.12 -> 4
    (6, 2, 0.5, 4),                   # 3 * 1.5 = 4.5 -> 4
    (5, 3, 0.5, 3),                   # ceil(5/3) = 2; 3.0
    (101, 4, 0.1, 28),                # ceil(25.25) = 26; 28.6 -> 28
])
def test_lmax_closed_form(total, k, eps, want):
    assert oracle.lmax(total, k, eps) == want


# --- hand-derived fixtures -------------------------------------------------------------

@pytest.mark.parametrize("g", GOLDEN, ids=[g.name for g in GOLDEN])
def test_golden_fixture(g):
    o = oracle.Oracle(g.n, g.m, g.net_off, g.pins, g.k, g.eps, g.part, g.vertex_w, g.net_w,
                      g.subrounds, g.seed)
    assert o.lmax == g.lmax
    assert o.objective() == g.objective
    for u, i, want in g.gains:
        assert o.gain(u, i) == want, (u, i)
    stats, _ = o.refine(len(g.rounds))
    assert [tuple(r) for r in stats.tolist()] == list(g.rounds)
    np.testing.assert_array_equal(o.partition(), g.final)


# --- P1: maintained state equals the definitions recomputed from Pi ----------------------

@pytest.mark.parametrize("seed", range(6))
def test_definitions_recomputed_every_round(seed):
    k = [2, 3, 4, 5, 8, 13][seed]
    hg = synth.random_small(seed, 60, 50, k, max_size=7, weighted=seed % 2 == 1, rounds=4)
    t = Tiny.from_hypergraph(hg)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=1 + seed % 4, seed=seed)
    sizes = np.diff(hg.net_off)
    for _ in range(4):
        stats, _ = o.refine(1)
        part = o.partition()
        phi = o.phi()
        np.testing.assert_array_equal(phi, t.phi(part))
        np.testing.assert_array_equal(phi.sum(axis=1), sizes)
        np.testing.assert_array_equal(o.block_weights(), t.block_weights(part))
        assert o.block_weights().sum() == sum(t.vw)
        assert o.objective() == t.objective(part) == stats[0, 0]
        assert stats[0, 4] == max(t.block_weights(part))


# --- P2: gain = objective reduction (brute force) ----------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_gain_equals_objective_difference(seed):
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(2, 6))
    t = random_tiny(rng, 12, 10, k, max_size=5, weighted=seed % 2 == 0)
    part = rng.integers(0, k, size=t.n)
    o = make_oracle(t, part)
    for u in range(t.n):
        for i in range(k):
            if i != part[u]:
                assert o.gain(u, i) == t.gain(part, u, i), (u, i)


# --- P3: graph special case (all nets of size 2) -----------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_graph_gain_is_edge_cut_gain(seed):
    rng = np.random.default_rng(200 + seed)
    n, k = 20, 3
    edges = set()
    while len(edges) < 40:
        a, b = rng.choice(n, size=2, replace=False)
        edges.add((int(min(a, b)), int(max(a, b))))
    edges = sorted(edges)
    w = rng.integers(1, 9, size=len(edges)).tolist()
    t = Tiny(n, [list(e) for e in edges], k, 0.3, None, w)
    part = rng.integers(0, k, size=n)
    o = make_oracle(t, part)
    for u in range(n):
        a = int(part[u])
        to_block = [0] * k
        for (x, y), we in zip(edges, w):
            if u in (x, y):
                v = y if x == u else x
                to_block[int(part[v])] += we
        for i in range(k):
            if i != a:
                # textbook graph gain: omega(u, V_i) - omega(u, V_a \ {u})
                assert o.gain(u, i) == to_block[i] - to_block[a]


# --- P4 + whole rounds: brute-force synchronous rounds and the replay invariant -----------

@pytest.mark.parametrize("seed", range(10))
def test_rounds_match_bruteforce(seed):
    rng = np.random.default_rng(300 + seed)
    k = int(rng.integers(2, 5))
    S = int(rng.integers(1, 5))
    t = random_tiny(rng, 14, 12, k, max_size=4, weighted=seed % 3 == 0, eps=0.3)
    part = rng.integers(0, k, size=t.n)
    o = make_oracle(t, part, S=S, seed=seed)
    stats, moves = o.refine(4, log_moves=True)
    want_part, want_stats, want_log, _ = lp_rounds(t, part, 4, S=S, seed=seed)
    assert [tuple(r) for r in stats.tolist()] == want_stats
    assert [tuple(m) for m in moves.tolist()] == want_log
    np.testing.assert_array_equal(o.partition(), want_part)


@pytest.mark.parametrize("seed", range(8))
def test_replay_invariant(seed):
    """Replaying each sub-round's moves one at a time (ascending id), the oracle's gain
    formula at the current state equals the realised objective change of that step, so the
    steps sum to the sub-round's change; a mover that shares no net with another mover of
    its sub-round realises exactly its frozen gain."""
    rng = np.random.default_rng(400 + seed)
    k = int(rng.integers(2, 5))
    t = random_tiny(rng, 16, 14, k, max_size=4, weighted=True, eps=0.4)
    part = [int(x) for x in rng.integers(0, k, size=t.n)]
    o = make_oracle(t, part, S=2, seed=seed)
    _, moves = o.refine(3, log_moves=True)
    cur = list(part)
    for sub in sorted(set(moves[:, 0].tolist())):
        mv = sorted((m for m in moves.tolist() if m[0] == sub), key=lambda m: m[1])
        frozen = make_oracle(t, cur)
        movers = {m[1] for m in mv}
        obj0, total = t.objective(cur), 0
        for _, u, a, b in mv:
            assert cur[u] == a
            g_now = make_oracle(t, cur).gain(u, b)
            before = t.objective(cur)
            cur[u] = b
            assert before - t.objective(cur) == g_now
            total += g_now
            if not any(v in movers and v != u for e in t.inc[u] for v in t.nets[e]):
                assert g_now == frozen.gain(u, b)
        assert obj0 - t.objective(cur) == total
    np.testing.assert_array_equal(o.partition(), cur)


# --- P5: exhaustive optimal bipartitions -------------------------------------------------

def _optimum(t: Tiny):
    lmax = t.lmax()
    best, arg = None, None
    for assign in itertools.product(range(t.k), repeat=t.n):
        if max(t.block_weights(assign)) > lmax:
            continue
        obj = t.objective(assign)
        if best is None or obj < best:
            best, arg = obj, list(assign)
    return best, arg


@pytest.mark.parametrize("seed,n,k", [(0, 10, 2), (1, 10, 2), (2, 9, 2), (3, 8, 3),
                                      (4, 10, 2), (5, 7, 3), (6, 12, 2), (7, 12, 2), (8, 11, 2)])
def test_exhaustive_optimum(seed, n, k):
    rng = np.random.default_rng(500 + seed)
    t = random_tiny(rng, n, n + 2, k, max_size=4, weighted=seed % 2 == 1, eps=0.25)
    opt, arg = _optimum(t)
    assert opt is not None
    # a balanced start refined by LP never beats the optimum over balanced partitions
    start = [v % k for v in range(n)]
    if max(t.block_weights(start)) <= t.lmax():
        o = make_oracle(t, start, S=2, seed=seed)
        o.refine(5)
        assert o.objective() >= opt
        assert max(o.block_weights()) <= t.lmax()
    # started at an optimum, no positive-gain feasible move exists, so LP moves nothing
    o = make_oracle(t, arg, S=3, seed=seed)
    stats, _ = o.refine(3)
    assert stats[:, 2].sum() == 0
    assert o.objective() == opt


# --- P6: balance -------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_balance_never_worsens(seed):
    rng = np.random.default_rng(600 + seed)
    k = int(rng.integers(2, 6))
    hg = synth.random_small(700 + seed, 80, 70, k, max_size=6, weighted=True, eps=0.05)
    # an unbalanced start: a third of the vertices piled into block 0
    part = hg.part.copy()
    part[rng.choice(hg.n, size=hg.n // 3, replace=False)] = 0
    o = oracle.Oracle.from_hypergraph(hg, subrounds=2, seed=seed, part=part)
    lm = o.lmax
    prev = o.block_weights()
    for _ in range(5):
        o.refine(1)
        w = o.block_weights()
        assert np.all(w <= np.maximum(prev, lm))
        assert np.all(w[prev <= lm] <= lm)
        prev = w


# --- empty nets, single-pin nets, isolated vertices --------------------------------------

def test_degenerate_nets():
    t = Tiny(5, [[], [0], [1, 2], [2, 3, 4], []], 2, 0.5, None, [3, 2, 4, 1, 5])
    part = [0, 1, 0, 1, 1]
    o = make_oracle(t, part, S=1)
    assert o.objective() == t.objective(part) == 4 + 1
    stats, moves = o.refine(3, log_moves=True)
    want_part, want_stats, want_log, _ = lp_rounds(t, part, 3, S=1)
    assert [tuple(r) for r in stats.tolist()] == want_stats
    np.testing.assert_array_equal(o.partition(), want_part)


def test_rejects_bad_partition():
    t = Tiny(3, [[0, 1]], 2, 0.1)
    off, pins = t.csr()
    with pytest.raises(ValueError):
        oracle.Oracle(3, 1, off, pins, 2, 0.1, np.array([0, 2, 1], np.int32))


# --- variant: zero-gain balance moves (Sec. 6) ----------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_balance_moves_match_bruteforce(seed):
    rng = np.random.default_rng(900 + seed)
    k = int(rng.integers(2, 5))
    S = int(rng.integers(1, 4))
    t = random_tiny(rng, 14, 12, k, max_size=4, weighted=seed % 2 == 0, eps=0.5)
    part = rng.integers(0, k, size=t.n)
    part[: t.n // 2] = 0                                  # unbalanced: balance moves matter
    off, pins = t.csr()
    vw = None if all(x == 1 for x in t.vw) else np.array(t.vw, dtype=np.int32)
    nw = None if all(x == 1 for x in t.nw) else np.array(t.nw, dtype=np.int32)
    o = oracle.Oracle(t.n, t.m, off, pins, k, t.eps, part.astype(np.int32), vw, nw, S, seed,
                      balance_moves=True)
    stats, moves = o.refine(4, log_moves=True)
    want_part, want_stats, want_log, _ = lp_rounds(t, part, 4, S=S, seed=seed, balance_moves=True)
    assert [tuple(r) for r in stats.tolist()] == want_stats
    assert [tuple(m) for m in moves.tolist()] == want_log
    np.testing.assert_array_equal(o.partition(), want_part)


def test_balance_moves_hand_example():
    # Nets {0,1} and {2,3}, all four vertices in block 0 (k = 2, eps = 0.5, c(V) = 4,
    # L_max = floor(1.5 * 2) = 3).  Every move cuts a net (gain -1), so there is neither a
    # positive- nor a zero-gain move, and nothing moves even with the variant.
    t = Tiny(4, [[0, 1], [2, 3]], 2, 0.5)
    o = make_oracle(t, [0, 0, 0, 0], S=1)
    o2 = oracle.Oracle(4, 2, *t.csr(), 2, 0.5, np.zeros(4, np.int32), None, None, 1, 0,
                       balance_moves=True)
    assert o2.refine(1)[0][0, 2] == 0
    # An isolated vertex has gain 0 to every block: with the variant it leaves the overloaded
    # block 0 (w0 = 4 > L_max = 3) for block 1, the only lighter block (0 + 1 < 4).
    t2 = Tiny(5, [[0, 1], [2, 3]], 2, 0.5)            # vertex 4 has no nets; c(V) = 5, L_max = 4
    o3 = oracle.Oracle(5, 2, *t2.csr(), 2, 0.5, np.zeros(5, np.int32), None, None, 1, 0,
                       balance_moves=True)
    st, mv = o3.refine(1, log_moves=True)
    assert [tuple(x) for x in mv.tolist()] == [(0, 4, 0, 1)]
    assert st[0, 0] == 0 and st[0, 2] == 1


def test_balance_moves_need_room():
    # k = 3, eps = 0, c(V) = 9, L_max = 3; blocks 0 = {0..4} (w 5), 1 = {5,6,7} (w 3),
    # 2 = {8} (w 1); one net {0, 1, 5}.  Vertices 0 and 1 have gain 0 to block 1 (Phi(e,0) = 2,
    # Phi(e,1) = 1) and 1 + 3 < 5, but block 1 has no room, and their gain to block 2 is -1:
    # no candidate.  Vertex 5 has gain +1 to the full block 0 and gain 0 to block 2 (1 + 1 < 3):
    # a balance candidate, like the isolated 2, 3, 4 (block 0) and 6, 7 (block 1), all for
    # block 2.  Block 2 has room for two: ids 2 and 3 (all gains 0).
    t = Tiny(9, [[0, 1, 5]], 3, 0.0)
    part = [0, 0, 0, 0, 0, 1, 1, 1, 2]
    assert t.lmax() == 3
    o = oracle.Oracle(9, 1, *t.csr(), 3, 0.0, np.array(part, np.int32), None, None, 1, 0,
                      balance_moves=True)
    st, mv = o.refine(1, log_moves=True)
    assert st[0].tolist() == [1, 6, 2, 9, 3]
    assert [tuple(x) for x in mv.tolist()] == [(0, 2, 0, 2), (0, 3, 0, 2)]
    _, want_stats, want_log, _ = lp_rounds(t, part, 1, S=1, balance_moves=True)
    assert want_stats == [(1, 6, 2, 9, 3)] and want_log == [(0, 2, 0, 2), (0, 3, 0, 2)]


# --- variant: revert of negative attributed gains (Sec. 5.2, Sec. 6) -----------------------

@pytest.mark.parametrize("seed", range(10))
def test_revert_matches_bruteforce(seed):
    rng = np.random.default_rng(950 + seed)
    k = int(rng.integers(2, 5))
    S = int(rng.integers(1, 3))
    t = random_tiny(rng, 14, 14, k, max_size=4, weighted=seed % 2 == 0, eps=0.6)
    part = rng.integers(0, k, size=t.n)
    off, pins = t.csr()
    vw = None if all(x == 1 for x in t.vw) else np.array(t.vw, dtype=np.int32)
    nw = None if all(x == 1 for x in t.nw) else np.array(t.nw, dtype=np.int32)
    balance = seed % 3 == 0
    o = oracle.Oracle(t.n, t.m, off, pins, k, t.eps, part.astype(np.int32), vw, nw, S, seed,
                      balance_moves=balance, revert_negative=True)
    stats, moves = o.refine(4, log_moves=True)
    rev = []
    want_part, want_stats, want_log, _ = lp_rounds(t, part, 4, S=S, seed=seed, balance_moves=balance,
                                                   revert_negative=True, reverted=rev)
    assert [tuple(r) for r in stats.tolist()] == want_stats
    assert [tuple(m) for m in moves.tolist()] == want_log
    assert o.reverted.tolist() == rev
    np.testing.assert_array_equal(o.partition(), want_part)


def test_revert_happens_on_random_tiny():
    # the brute-force comparison above must include sub-rounds with reverts
    total = 0
    for seed in range(40):
        rng = np.random.default_rng(3000 + seed)
        t = random_tiny(rng, 12, 12, 2, max_size=3, eps=0.6)
        rev = []
        lp_rounds(t, rng.integers(0, 2, size=t.n), 2, S=1, seed=seed, revert_negative=True, reverted=rev)
        total += sum(rev)
    assert total > 0


def test_revert_hand_example_swap():
    # Net {0,1} of weight 5 with vertex 0 in block 0 and vertex 1 in block 1; vertices 2 and
    # 3 are isolated padding (c(V) = 4, L_max = floor(1.5 * 2) = 3).  Both 0 -> 1 and 1 -> 0
    # have gain 5 against the frozen state and both fit, so both are approved (S = 1).  In id
    # order, 0 -> 1 first removes the cut (+5); then 1 -> 0 cuts the net again (-5), so the
    # move of vertex 1 is reverted: the net ends up uncut in block 1 (weight 3 = L_max).
    t = Tiny(4, [[0, 1]], 2, 0.5, None, [5])
    part = [0, 1, 0, 1]
    plain = make_oracle(t, part, S=1)
    st_plain, _ = plain.refine(1)
    assert st_plain[0].tolist() == [5, 2, 2, 4, 2]             # the swap keeps the cut
    o = oracle.Oracle(4, 1, *t.csr(), 2, 0.5, np.array(part, np.int32), None,
                      np.array([5], np.int32), 1, 0, revert_negative=True)
    st, mv = o.refine(1, log_moves=True)
    assert st[0].tolist() == [0, 2, 2, 4, 3]
    assert o.reverted.tolist() == [1]
    assert [tuple(x) for x in mv.tolist()] == [(0, 0, 0, 1), (0, 1, 1, 0), (0, 1, 0, 1)]
    assert o.partition().tolist() == [1, 1, 0, 1]
    # eligibility: the reverted vertex counts as moved, so round 1 sees all vertices of the net
    st1, _ = o.refine(1)
    assert st1[0, 3] == 2


def test_revert_attributed_gains_sum_to_objective_change():
    # Sec. 5.2: the attributed gains of a sub-round's moves add up to the objective it removed;
    # here the attributed gains are the exact gains of the id-ordered sequence (Sec. 5.4)
    rng = np.random.default_rng(77)
    for seed in range(6):
        t = random_tiny(rng, 16, 14, 3, max_size=4, weighted=True, eps=0.6)
        part = rng.integers(0, 3, size=t.n)
        o = make_oracle(t, part, S=1)
        before = o.objective()
        _, log = o.refine(1, log_moves=True)
        if len(log) == 0:
            continue
        gains = make_oracle(t, part, S=1).exact_gains(log[:, 1:4])
        assert int(gains.sum()) == before - o.objective()
