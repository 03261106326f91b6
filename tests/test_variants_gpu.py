"""GPU parity of the LP variants of Sec. 6 against the oracle (bit-exact, all integer).

* balance moves: a vertex without a feasible positive-gain target may take a zero-gain move
  to the lightest block t with room and w(t) + c(u) < w(Pi(u)).
* revert: after each sub-round, the moves whose attributed gain (every net seeing the moves
  in ascending vertex id, Sec. 5.2 / Lemma 1) is negative are undone.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2010_10272_gb300 import HGP
from parity_util import compare_state, run_both

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import build as b
    b.build()
    oracle.build()


BALANCE_CASES = [
    # (seed, n, m, k, max_size, weighted, S, phi_width, eps)
    (1, 5000, 3000, 2, 4, False, 4, 0, 0.03),
    (2, 7001, 5000, 3, 6, True, 1, 0, 0.05),
    (3, 6143, 4000, 8, 5, False, 4, 0, 0.03),
    (4, 9999, 8000, 16, 10, True, 7, 2, 0.1),
    (5, 4097, 2000, 32, 4, False, 2, 4, 0.03),
    (6, 6000, 5500, 33, 9, True, 4, 1, 0.03),
    (7, 8191, 7000, 64, 12, True, 5, 0, 0.05),
    (8, 2049, 2500, 5, 300, True, 4, 1, 0.03),    # wide tier
]


@pytest.mark.parametrize("case", BALANCE_CASES, ids=[f"s{c[0]}-k{c[3]}-S{c[6]}" for c in BALANCE_CASES])
def test_balance_moves_random(case):
    seed, n, m, k, max_size, weighted, S, w, eps = case
    hg = synth.random_small(100 + seed, n, m, k, max_size=max_size, weighted=weighted, eps=eps, rounds=4)
    part = hg.part.copy()
    part[: n // 3] = 0           # an unbalanced start, so zero-gain moves have work to do
    h, o, stats = run_both(hg, rounds=4, S=S, seed=seed, phi_width=w, part=part, balance_moves=True)
    # the variant differs from the plain rule on these inputs
    h0, _, stats0 = run_both(hg, rounds=4, S=S, seed=seed, phi_width=w, part=part)
    assert not np.array_equal(h.partition(), h0.partition())


def test_balance_moves_isolated_and_heavy_vertices():
    # isolated vertices have gain 0 everywhere; heavy nets (W > 2047) take the cooperative path
    rng = np.random.default_rng(5)
    hg = synth.random_small(55, 6000, 3000, 8, max_size=6, weighted=True, eps=0.05, rounds=3)
    hg.net_w = rng.integers(1, 2000, size=hg.m, dtype=np.int32)
    part = hg.part.copy()
    part[: hg.n // 2] = 3
    run_both(hg, rounds=3, S=3, seed=2, part=part, balance_moves=True)


@pytest.mark.parametrize("k,S", [(4, 2), (64, 3)])
def test_balance_candidates_match_oracle(k, S):
    hg = synth.random_small(70 + k, 9000, 6000, k, max_size=6, weighted=True, eps=0.04)
    part = hg.part.copy()
    part[: hg.n // 3] = 1
    h = HGP.from_hypergraph(hg, part=part, subrounds=S, seed=3, balance_moves=True)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=3, part=part, balance_moves=True)
    zero = 0
    for step in range(2):
        for s in range(S):
            t_h, g_h = h.debug_candidates(s)
            t_o, g_o = o.candidates(s)
            np.testing.assert_array_equal(t_h, t_o)
            np.testing.assert_array_equal(g_h, g_o)
            zero += int(((t_o >= 0) & (g_o == 0)).sum())
        h.refine(1)
        o.refine(1)
    assert zero > 0


def test_balance_moves_powerlaw_scaled():
    hg = synth.config_powerlaw(scale=0.002)
    part = hg.part.copy()
    part[: hg.n // 4] = 0
    run_both(hg, rounds=3, S=4, part=part, check_phi=False, balance_moves=True)


# ---------------------------------------------------------------- revert of negative moves
REVERT_CASES = [
    # (seed, n, m, k, max_size, weighted, S, phi_width, eps)
    (1, 5000, 3000, 2, 4, False, 1, 0, 0.03),
    (2, 7001, 5000, 3, 6, True, 1, 0, 0.05),
    (3, 6143, 4000, 8, 5, False, 2, 0, 0.03),
    (4, 9999, 8000, 16, 10, True, 4, 2, 0.1),
    (5, 4097, 2000, 32, 4, False, 1, 4, 0.03),
    (6, 6000, 5500, 33, 9, True, 4, 1, 0.03),
    (7, 8191, 7000, 64, 12, True, 1, 0, 0.05),
    (8, 2049, 2500, 5, 300, True, 1, 1, 0.03),    # wide tier
]


def _run_revert(hg, rounds, S, seed, phi_width=0, balance=False, graph=0, check_phi=True):
    h = HGP.from_hypergraph(hg, subrounds=S, seed=seed, phi_width=phi_width, graph=graph,
                            revert_negative=True, balance_moves=balance)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=seed, revert_negative=True,
                                      balance_moves=balance)
    got = h.refine(rounds)
    want, _ = o.refine(rounds)
    np.testing.assert_array_equal(got[:, :5], want)
    np.testing.assert_array_equal(got[:, 6], o.reverted)
    compare_state(h, o, check_phi)
    return h, o, got


@pytest.mark.parametrize("balance", [False, True])
@pytest.mark.parametrize("case", REVERT_CASES, ids=[f"s{c[0]}-k{c[3]}-S{c[6]}" for c in REVERT_CASES])
def test_revert_random(case, balance):
    seed, n, m, k, max_size, weighted, S, w, eps = case
    hg = synth.random_small(200 + seed, n, m, k, max_size=max_size, weighted=weighted, eps=eps, rounds=4)
    _run_revert(hg, 4, S, seed, phi_width=w, balance=balance)


def test_revert_happens_and_graph_replay():
    hg = synth.random_small(204, 9999, 8000, 16, max_size=10, weighted=True, eps=0.1, rounds=4)
    h, o, got = _run_revert(hg, 4, 4, 4, phi_width=2, graph=1)
    assert got[:, 6].sum() > 100
    # a second call replays the captured graph
    got2 = h.refine(4)
    want2, _ = o.refine(4)
    np.testing.assert_array_equal(got2[:, :5], want2)
    np.testing.assert_array_equal(got2[:, 6], o.reverted)
    compare_state(h, o)


def test_revert_hand_example_swap():
    # net {0,1} (omega 5), vertex 0 in block 0, vertex 1 in block 1, isolated padding 2, 3: the
    # swap is approved, and the move of vertex 1 (attributed gain -5 after 0 -> 1) is undone
    h = HGP(4, 1, np.array([0, 2], np.int64), np.array([0, 1], np.int32), 2, 0.5,
            np.array([0, 1, 0, 1], np.int32), None, np.array([5], np.int32), subrounds=1,
            revert_negative=True)
    st = h.refine(1)
    assert st[0, :5].tolist() == [0, 2, 2, 4, 3] and st[0, 6] == 1
    assert h.partition().tolist() == [1, 1, 0, 1]


def test_revert_powerlaw_scaled():
    hg = synth.config_powerlaw(scale=0.002)
    _run_revert(hg, 3, 4, 0, check_phi=False)


def test_revert_rejected_in_batch():
    from paper_2010_10272_gb300 import Batch, HGPError
    hg = synth.random_small(5, 3000, 2000, 4, rounds=2)
    a = HGP.from_hypergraph(hg)
    b = HGP.from_hypergraph(hg, revert_negative=True)
    with pytest.raises(HGPError):
        Batch([a, b])


def test_revert_profile_phase():
    hg = synth.random_small(36, 20000, 18000, 8, max_size=9, weighted=True, rounds=3)
    h = HGP.from_hypergraph(hg, subrounds=4, revert_negative=True)
    h.set_profiling(True)
    l0 = h.launch_count()
    h.refine(3)
    launched = h.launch_count() - l0
    prof = h.profile()
    assert sum(v[1] for v in prof.values()) == launched
    assert prof["revert"][1] == 3 * 4 * 4 and prof["revert"][0] > 0
