"""Pins for the oracle's two candidate routines, which the full-size GPU checks rely on.

* ``Oracle.candidates`` (the candidates of one sub-round of the next round against the
  current state) is compared with brute-force candidates: gains as objective reductions,
  eligibility from the neighbourhoods of the vertices moved in the previous round (Sec. 6),
  the sub-round from the published SplitMix64 output function.
* ``oracle.sample_candidates`` (round-0 candidates of sampled vertices, with pin counts
  taken from the pins of each net touching the sample instead of a Phi table) is compared
  with the same brute force on tiny inputs, and with ``Oracle.candidates`` on larger ones.
Nothing here compares the oracle with itself through a shared formula, and nothing reads
the CUDA library.
"""
import types

import numpy as np
import pytest

import oracle
import synth
from brute import candidates, eligible_after, lp_rounds, random_tiny


def _oracle(t, part, S, seed):
    off, pins = t.csr()
    vw = None if all(x == 1 for x in t.vw) else np.array(t.vw, dtype=np.int32)
    nw = None if all(x == 1 for x in t.nw) else np.array(t.nw, dtype=np.int32)
    return oracle.Oracle(t.n, t.m, off, pins, t.k, t.eps, np.array(part, dtype=np.int32), vw, nw,
                         S, seed)


def _as_hypergraph(t, part):
    off, pins = t.csr()
    return types.SimpleNamespace(
        n=t.n, m=t.m, k=t.k, eps=t.eps, net_off=off, pins=pins, part=np.asarray(part, np.int32),
        vertex_w=None if all(x == 1 for x in t.vw) else np.array(t.vw, dtype=np.int32),
        net_w=None if all(x == 1 for x in t.nw) else np.array(t.nw, dtype=np.int32))


def _dense(cands, n):
    tg = np.full(n, -1, np.int32)
    g = np.zeros(n, np.int64)
    for u, (i, gain) in cands.items():
        tg[u], g[u] = i, gain
    return tg, g


@pytest.mark.parametrize("seed", range(12))
def test_candidates_match_bruteforce_after_rounds(seed):
    """Sub-round filter, eligibility and best target of the next round, after 0-2 rounds."""
    rng = np.random.default_rng(900 + seed)
    k = int(rng.integers(2, 5))
    S = int(rng.integers(1, 4))
    t = random_tiny(rng, 13, 11, k, max_size=4, weighted=seed % 2 == 1, eps=0.3)
    part0 = rng.integers(0, k, size=t.n)
    rounds = seed % 3
    o = _oracle(t, part0, S, seed)
    o.refine(rounds)
    part, _, _, moved = lp_rounds(t, part0, rounds, S=S, seed=seed)
    np.testing.assert_array_equal(o.partition(), part)
    elig = eligible_after(t, moved if rounds else None)
    if rounds:
        assert len(elig) < t.n or not moved or all(t.inc[v] for v in moved)
    seen = 0
    for s in range(S):
        want_t, want_g = _dense(candidates(t, part, elig, rounds, s, S, seed), t.n)
        got_t, got_g = o.candidates(s)
        np.testing.assert_array_equal(got_t, want_t)
        np.testing.assert_array_equal(got_g, want_g)
        seen += int((want_t >= 0).sum())
    assert o.round == rounds


def test_candidates_see_only_eligible_vertices():
    """Hand example (k = 2, S = 1, unit weights, eps = 0.5): nets {0,1} and {2,3}, start
    partition [0, 1, 1, 0].  L_max = floor(1.5 * 2) = 3, so each block has room for one more
    vertex.  Round 0: every vertex has gain 1 (leaving makes its net uncut); per target block
    the smaller id wins the single slot, so 0 -> 1 and 1 -> 0 (a synchronous swap, net {0,1}
    stays cut) and the partition becomes [1, 0, 1, 0].  Round 1: only the vertices sharing a
    net with a moved vertex, 0 and 1, are eligible; 2 and 3 still have gain 1 but are not."""
    from brute import Tiny
    t = Tiny(4, [[0, 1], [2, 3]], 2, 0.5)
    part = [0, 1, 1, 0]
    o = _oracle(t, part, 1, 0)
    got_t, got_g = o.candidates(0)
    np.testing.assert_array_equal(got_t, [1, 0, 0, 1])
    np.testing.assert_array_equal(got_g, [1, 1, 1, 1])
    o.refine(1)
    np.testing.assert_array_equal(o.partition(), [1, 0, 1, 0])
    got_t, got_g = o.candidates(0)
    np.testing.assert_array_equal(got_t, [0, 1, -1, -1])
    np.testing.assert_array_equal(got_g, [1, 1, 0, 0])
    # the brute force agrees
    _, _, _, moved = lp_rounds(t, part, 1, S=1, seed=0)
    assert moved == {0, 1}
    want_t, _ = _dense(candidates(t, [1, 0, 1, 0], eligible_after(t, moved), 1, 0, 1), 4)
    np.testing.assert_array_equal(got_t, want_t)


@pytest.mark.parametrize("seed", range(16))
def test_sample_candidates_match_bruteforce(seed):
    rng = np.random.default_rng(1300 + seed)
    k = int(rng.integers(2, 6))
    S = int(rng.integers(1, 5))
    t = random_tiny(rng, 15, 14, k, max_size=5, weighted=seed % 2 == 0, eps=0.25)
    part = rng.integers(0, k, size=t.n)
    hg = _as_hypergraph(t, part)
    sample = rng.permutation(t.n)[: int(rng.integers(1, t.n + 1))].astype(np.int32)
    for s in range(S):
        want_t, want_g = _dense(candidates(t, list(part), set(range(t.n)), 0, s, S, seed), t.n)
        got_t, got_g = oracle.sample_candidates(hg, sample, s=s, subrounds=S, seed=seed)
        np.testing.assert_array_equal(got_t, want_t[sample])
        np.testing.assert_array_equal(got_g, want_g[sample])


@pytest.mark.parametrize("weighted,k,S", [(False, 2, 4), (True, 7, 3), (True, 33, 2), (False, 64, 4)])
def test_sample_candidates_match_full_oracle(weighted, k, S):
    hg = synth.random_small(41 + k, 4000, 3500, k, max_size=12, weighted=weighted)
    rng = np.random.default_rng(k)
    sample = rng.choice(hg.n, size=700, replace=False).astype(np.int32)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=3)
    found = 0
    for s in range(S):
        full_t, full_g = o.candidates(s)
        got_t, got_g = oracle.sample_candidates(hg, sample, s=s, subrounds=S, seed=3)
        np.testing.assert_array_equal(got_t, full_t[sample])
        np.testing.assert_array_equal(got_g, full_g[sample])
        found += int((got_t >= 0).sum())
    assert found > 20


@pytest.mark.parametrize("threads", [2, 5])
def test_threads_do_not_change_results(threads):
    """The candidate step split over threads gives the sequential oracle's rounds exactly
    (n above the size from which the slices are used)."""
    hg = synth.random_small(77, 9000, 8000, 6, max_size=9, weighted=True)
    a = oracle.Oracle.from_hypergraph(hg, subrounds=3, seed=2)
    b = oracle.Oracle.from_hypergraph(hg, subrounds=3, seed=2, threads=threads)
    sa, ma = a.refine(4, log_moves=True)
    sb, mb = b.refine(4, log_moves=True)
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(a.phi(), b.phi())
    np.testing.assert_array_equal(a.phi_rows(100, 250), a.phi()[100:250].astype(np.int32))
    assert sa[:, 2].sum() > 100
