"""GPU parity of rebalancing (Sec. 8, synchronous reading) against the oracle: per-pass
statistics, phases, partition, Phi, Lambda, block weights and objective, bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from paper_2010_10272_gb300 import HGP, HGPError
from parity_util import compare_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import build as b
    b.build()
    oracle.build()


def _both(hg, part, S, seed, passes=12, phi_width=0, check_phi=True):
    h = HGP.from_hypergraph(hg, part=part, subrounds=S, seed=seed, phi_width=phi_width)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=seed, part=part)
    st, ph = h.rebalance(passes)
    want, want_ph, log = o.rebalance(passes, log_moves=True)
    np.testing.assert_array_equal(ph, want_ph)
    np.testing.assert_array_equal(st[:, :5], want)
    deg = np.diff(hg.net_off)
    vdeg = np.bincount(hg.pins, minlength=hg.n)
    S_ = S
    for i in range(st.shape[0]):
        sel = log[(log[:, 0] // S_) == i]
        assert st[i, 5] == vdeg[sel[:, 1]].sum()
    assert np.all(st[:, 6] == 0)
    compare_state(h, o, check_phi)
    del deg
    return h, o, st, ph


CASES = [
    # (seed, n, m, k, max_size, weighted, S, phi_width, eps, skew)
    (1, 5000, 4000, 2, 6, False, 4, 0, 0.03, 0.5),
    (2, 7001, 6000, 3, 8, True, 1, 0, 0.05, 0.6),
    (3, 6143, 5000, 8, 6, False, 4, 0, 0.03, 0.4),
    (4, 9999, 8000, 16, 10, True, 3, 2, 0.1, 0.5),
    (5, 4097, 3000, 32, 5, False, 2, 4, 0.03, 0.3),
    (6, 6000, 5500, 33, 9, True, 4, 1, 0.03, 0.5),
    (7, 8191, 7000, 64, 12, True, 2, 0, 0.05, 0.2),
    (8, 2049, 2500, 5, 300, True, 2, 1, 0.03, 0.5),     # wide tier
]


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-k{c[3]}-S{c[6]}" for c in CASES])
def test_rebalance_random(case):
    seed, n, m, k, max_size, weighted, S, w, eps, skew = case
    hg = synth.random_small(300 + seed, n, m, k, max_size=max_size, weighted=weighted, eps=eps)
    part = hg.part.copy()
    part[: int(n * skew)] = 0
    h, o, st, ph = _both(hg, part, S, seed, phi_width=w)
    assert st.shape[0] >= 1 and st[:, 2].sum() > 0


def test_phase_two_with_large_gains():
    # net weights up to 2^20: phase-2 priorities (gain + W_max) need the refinement levels
    rng = np.random.default_rng(21)
    hg = synth.random_small(321, 6000, 7000, 4, max_size=5, eps=0.01)
    hg.net_w = rng.integers(1, 1 << 20, size=hg.m, dtype=np.int32)
    part = hg.part.copy()
    part[: hg.n * 2 // 3] = 0
    h, o, st, ph = _both(hg, part, 2, 3)
    assert 2 in ph.tolist()


def test_hand_example_path():
    h = HGP(6, 5, np.array([0, 2, 4, 6, 8, 10], np.int64),
            np.array([0, 1, 1, 2, 2, 3, 3, 4, 4, 5], np.int32), 2, 1e-4, np.zeros(6, np.int32),
            subrounds=1)                      # L_max = floor(1.0001 * 3) = 3, as with eps = 0
    assert h.info()["lmax"] == 3
    st, ph = h.rebalance(5)
    assert ph.tolist() == [1, 2]
    assert st[:, :5].tolist() == [[0, 0, 0, 6, 6], [2, 6, 3, 6, 3]]
    assert h.partition().tolist() == [1, 1, 0, 0, 0, 1]
    st2, ph2 = h.rebalance(5)
    assert st2.shape[0] == 0


def test_refine_rebalance_refine():
    # rebalancing between LP rounds leaves the LP eligibility and round numbering untouched
    hg = synth.random_small(330, 9000, 8000, 8, max_size=8, weighted=True, eps=0.03)
    part = hg.part.copy()
    part[: hg.n // 2] = 5
    for graph in (0, 1):
        h = HGP.from_hypergraph(hg, part=part, subrounds=3, seed=2, graph=graph)
        o = oracle.Oracle.from_hypergraph(hg, subrounds=3, seed=2, part=part)
        np.testing.assert_array_equal(h.refine(2)[:, :5], o.refine(2)[0])
        st, ph = h.rebalance(10)
        want, want_ph, _ = o.rebalance(10)
        np.testing.assert_array_equal(st[:, :5], want)
        np.testing.assert_array_equal(ph, want_ph)
        np.testing.assert_array_equal(h.refine(3)[:, :5], o.refine(3)[0])
        compare_state(h, o)


def test_balanced_input_and_errors():
    hg = synth.random_small(331, 3000, 2000, 4, eps=0.05)
    h = HGP.from_hypergraph(hg)
    st, ph = h.rebalance(5)
    assert st.shape[0] == 0 and ph.shape[0] == 0
    with pytest.raises(HGPError):
        h.rebalance(-1)


def test_rebalance_powerlaw_scaled():
    hg = synth.config_powerlaw(scale=0.002)
    part = hg.part.copy()
    part[: hg.n // 3] = 0
    _both(hg, part, 4, 0, passes=8, check_phi=False)
