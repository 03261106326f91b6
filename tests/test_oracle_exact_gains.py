"""Pins for the oracle's exact gains of a move sequence (paper Sec. 5.4): brute force on tiny
inputs (objective differences along the sequence), the move sequences of LP sub-rounds
(their sum equals the objective change), and invalid sequences are rejected."""
import numpy as np
import pytest

import oracle
import synth
from brute import Tiny, random_tiny


def make(t, part):
    off, pins = t.csr()
    vw = None if all(x == 1 for x in t.vw) else np.array(t.vw, dtype=np.int32)
    nw = None if all(x == 1 for x in t.nw) else np.array(t.nw, dtype=np.int32)
    return oracle.Oracle(t.n, t.m, off, pins, t.k, t.eps, np.array(part, dtype=np.int32), vw, nw, 2, 0)


@pytest.mark.parametrize("seed", range(10))
def test_exact_gains_are_objective_differences(seed):
    rng = np.random.default_rng(800 + seed)
    k = int(rng.integers(2, 6))
    t = random_tiny(rng, 15, 14, k, max_size=5, weighted=seed % 2 == 0)
    part = [int(x) for x in rng.integers(0, k, size=t.n)]
    order = rng.permutation(t.n)[: int(rng.integers(1, t.n))]
    moves = []
    for u in order:
        b = int(rng.integers(0, k - 1))
        b = b + 1 if b >= part[u] else b
        moves.append((int(u), part[u], b))
    o = make(t, part)
    got = o.exact_gains(moves)
    cur = list(part)
    for j, (u, a, b) in enumerate(moves):
        before = t.objective(cur)
        cur[u] = b
        assert got[j] == before - t.objective(cur), j
    # the oracle's own state is untouched
    np.testing.assert_array_equal(o.partition(), part)


def test_lp_subround_gains_sum_to_objective_change():
    hg = synth.random_small(61, 400, 380, 4, max_size=6, weighted=True, rounds=3)
    t = Tiny.from_hypergraph(hg)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=2)
    part = o.partition()
    obj0 = o.objective()
    _, log = o.refine(1, log_moves=True)
    first = log[log[:, 0] == log[0, 0]]
    mv = [(int(u), int(a), int(b)) for _, u, a, b in first]
    o2 = make(t, part)
    g = o2.exact_gains(mv)
    cur = [int(x) for x in part]
    for u, a, b in mv:
        cur[u] = b
    assert obj0 - t.objective(cur) == g.sum()


def test_invalid_sequences_rejected():
    t = Tiny(4, [[0, 1], [1, 2, 3]], 2, 0.5)
    o = make(t, [0, 0, 1, 1])
    for bad in ([(0, 1, 0)], [(0, 0, 0)], [(0, 0, 1), (0, 1, 0)], [(9, 0, 1)], [(2, 1, 2)]):
        with pytest.raises(ValueError):
            o.exact_gains(bad)
