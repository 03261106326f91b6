"""Pins for the oracle's rebalancing (Sec. 8, synchronous reading): brute force on tiny inputs
(gains as objective differences), a hand-derived example, and invariants."""
import numpy as np
import pytest

import oracle
import synth
from brute import Tiny, lp_rounds, random_tiny, rebalance


def _oracle(t: Tiny, part, S, seed=0):
    off, pins = t.csr()
    vw = None if all(x == 1 for x in t.vw) else np.array(t.vw, dtype=np.int32)
    nw = None if all(x == 1 for x in t.nw) else np.array(t.nw, dtype=np.int32)
    return oracle.Oracle(t.n, t.m, off, pins, t.k, t.eps, np.array(part, dtype=np.int32), vw, nw, S, seed)


def test_hand_example_path():
    # Path 0-1-2-3-4-5 (unit nets), k = 2, eps = 0: c(V) = 6, L_max = 3; all in block 0.
    # Every move to block 1 cuts nets (gain -1 for the ends, -2 inside), so the phase-1 pass
    # has no candidate and phase 2 starts.  Order (gain desc, id asc): 0, 5, 1, 2, 3, 4; block 0
    # must shed 3: 0 (0 left before it), 5 (1), 1 (2) are selected, 2 (3) is not; block 1 has
    # room for 3.  Result [1,1,0,0,0,1]: nets {1,2} and {4,5} cut, objective 2.
    t = Tiny(6, [[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]], 2, 0.0)
    o = _oracle(t, [0] * 6, S=1)
    st, ph, mv = o.rebalance(5, log_moves=True)
    assert ph.tolist() == [1, 2]
    assert st.tolist() == [[0, 0, 0, 6, 6], [2, 6, 3, 6, 3]]
    assert [tuple(x) for x in mv.tolist()] == [(1, 0, 0, 1), (1, 1, 0, 1), (1, 5, 0, 1)]
    assert o.partition().tolist() == [1, 1, 0, 0, 0, 1]
    # balanced now: another call makes no pass
    st2, ph2, _ = o.rebalance(5)
    assert st2.shape[0] == 0 and ph2.shape[0] == 0


def test_hand_example_non_negative_first():
    # Nets {0, 4} and {1, 2}; blocks 0 = {0,1,2,3} (w 4), 1 = {4} (w 1); k = 2, eps = 0, c(V) = 5,
    # L_max = 3.  Phase 1: vertex 0 has gain +1 (joins 4), vertex 3 (isolated) gain 0, vertices
    # 1 and 2 gain -1.  Order 0, 3; block 0 sheds 1: only vertex 0 is selected.
    t = Tiny(5, [[0, 4], [1, 2]], 2, 0.0)
    o = _oracle(t, [0, 0, 0, 0, 1], S=1)
    st, ph, mv = o.rebalance(5, log_moves=True)
    assert ph.tolist() == [1]
    assert st.tolist() == [[0, 2, 1, 4, 3]]
    assert [tuple(x) for x in mv.tolist()] == [(0, 0, 0, 1)]


def test_hand_example_single_phase_one_sweep():
    # Path 0-1-2-3 (unit nets) and isolated 4, all in block 0; k = 2, eps = 0, c(V) = 5,
    # L_max = 3.  Pass 0 (phase 1): only vertex 4 has a non-negative gain (0) and moves; block
    # 0 still weighs 4.  Phase 1 is one sweep, so pass 1 is phase 2: gains -1 (ends 0, 3) and -2
    # (1, 2); order 0, 3, 1, 2; block 0 sheds 1: vertex 0 moves, cutting net {0,1}.
    t = Tiny(5, [[0, 1], [1, 2], [2, 3]], 2, 0.0)
    o = _oracle(t, [0] * 5, S=1)
    st, ph, mv = o.rebalance(5, log_moves=True)
    assert ph.tolist() == [1, 2]
    assert st.tolist() == [[0, 1, 1, 5, 4], [1, 4, 1, 4, 3]]
    assert [tuple(x) for x in mv.tolist()] == [(0, 4, 0, 1), (1, 0, 0, 1)]


@pytest.mark.parametrize("seed", range(12))
def test_matches_bruteforce(seed):
    rng = np.random.default_rng(1200 + seed)
    k = int(rng.integers(2, 5))
    S = int(rng.integers(1, 4))
    t = random_tiny(rng, 14, 12, k, max_size=4, weighted=seed % 2 == 0, eps=float(rng.choice([0.0, 0.1, 0.3])))
    part = rng.integers(0, k, size=t.n)
    part[: t.n // 2] = 0                                   # overloaded block 0
    o = _oracle(t, part, S=S, seed=seed)
    st, ph, mv = o.rebalance(6, log_moves=True)
    want_part, want_stats, want_ph, want_log = rebalance(t, part, 6, S=S, seed=seed)
    assert [tuple(r) for r in st.tolist()] == want_stats
    assert ph.tolist() == want_ph
    assert [tuple(m) for m in mv.tolist()] == want_log
    np.testing.assert_array_equal(o.partition(), want_part)
    np.testing.assert_array_equal(o.phi(), t.phi(want_part))


def test_no_eligibility_marks():
    # LP rounds, rebalancing, LP rounds: the rebalancing moves do not make vertices eligible
    moved_total = 0
    for seed in range(6):
        rng = np.random.default_rng(500 + seed)
        t = random_tiny(rng, 16, 14, 3, max_size=4, weighted=True, eps=0.05)
        part = rng.integers(0, 3, size=t.n)
        part[: 2 * t.n // 3] = 0                      # block 0 stays overloaded after LP
        moved_total += _lp_rebalance_lp(t, part, seed)
    assert moved_total > 0


def _lp_rebalance_lp(t, part, seed):
    o = _oracle(t, part, S=2, seed=seed)
    o.refine(2)
    p1, _, _, moved = lp_rounds(t, part, 2, S=2, seed=seed)
    _, _, mv = o.rebalance(4, log_moves=True)
    p2, _, _, log = rebalance(t, p1, 4, S=2, seed=seed)
    assert [tuple(m) for m in mv.tolist()] == log
    st, _ = o.refine(2)
    p3, want, _, _ = lp_rounds(t, p2, 2, S=2, seed=seed, start_round=2, moved_prev=moved)
    assert [tuple(r) for r in st.tolist()] == want
    np.testing.assert_array_equal(o.partition(), p3)
    return len(log)


@pytest.mark.parametrize("seed", range(4))
def test_invariants_random_small(seed):
    hg = synth.random_small(1300 + seed, 3000, 2500, [2, 4, 8, 16][seed], max_size=6,
                            weighted=seed % 2 == 1, eps=0.03)
    part = hg.part.copy()
    part[: hg.n // 2] = 0
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4, seed=seed, part=part)
    lm = o.lmax
    w0 = o.block_weights()
    st, ph, mv = o.rebalance(20, log_moves=True)
    assert st.shape[0] >= 1
    heaviest = np.concatenate([[w0.max()], st[:, 4]])
    assert np.all(np.diff(heaviest) <= 0)                    # the heaviest block never grows
    w = o.block_weights()
    assert np.all(w[w0 <= lm] <= lm)                          # no block becomes overloaded
    assert w.max() <= lm                                      # unit/small weights: balanced
    assert ph[0] == 1 and np.all(np.diff(ph) >= 0)
    # every move leaves an overloaded block for one with room
    assert np.all(w0[mv[:, 2]] > lm) or mv.shape[0] == 0


def test_balanced_input_makes_no_pass():
    hg = synth.random_small(7, 2000, 1500, 4, eps=0.05)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4)
    assert o.block_weights().max() <= o.lmax
    st, ph, mv = o.rebalance(5, log_moves=True)
    assert st.shape[0] == 0 and mv.shape[0] == 0
