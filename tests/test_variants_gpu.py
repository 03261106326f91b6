"""GPU parity of the LP variants of Sec. 6 against the oracle (bit-exact, all integer).

* balance moves: a vertex without a feasible positive-gain target may take a zero-gain move
  to the lightest block t with room and w(t) + c(u) < w(Pi(u)).
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2010_10272_gb300 import HGP
from parity_util import run_both

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
