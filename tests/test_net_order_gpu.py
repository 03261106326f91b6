"""Internal net order: nets relabelled by size class (largest first) inside the handle.

The order is an internal layout (records, Phi rows, pins in internal order; the incidence lists
carry internal ids), chosen by default from 2^20 nets on.  debug bit 2 forces it at small sizes
and bit 3 keeps the input order, so both layouts are checked here against the oracle: rounds,
partition, Phi and Lambda (returned in input net order), objective, the LP variants,
rebalancing, exact gains, checkpoints across layouts and batches.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import compare_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REORDER, KEEP = 4, 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import build as b
    b.build()
    oracle.build()


CASES = [
    # (seed, n, m, k, max_size, weighted, S, phi_width)
    (1, 5000, 4000, 2, 6, False, 4, 0),
    (4, 9999, 8000, 16, 10, True, 7, 2),
    (8, 8191, 7000, 64, 12, True, 5, 0),
    (10, 2049, 2500, 5, 300, True, 4, 1),    # nets > 255 pins -> wide tier with 1-byte Phi
]


@pytest.mark.parametrize("debug", [REORDER, REORDER | 2], ids=["direct", "bucketed"])
@pytest.mark.parametrize("case", CASES, ids=["k2", "k16-w2", "k64", "wide"])
def test_reordered_matches_oracle(case, debug):
    from paper_2010_10272_gb300 import HGP
    seed, n, m, k, max_size, weighted, S, w = case
    hg = synth.random_small(seed, n, m, k, max_size=max_size, weighted=weighted, rounds=4)
    h = HGP.from_hypergraph(hg, subrounds=S, seed=seed, phi_width=w, debug=debug | 1)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=S, seed=seed)
    compare_state(h, o)
    np.testing.assert_array_equal(h.refine(4)[:, :5], o.refine(4)[0])
    compare_state(h, o)


def test_skewed_sizes_both_layouts_identical():
    """A power-law instance (where the order differs most from the input's): both layouts give
    the same rounds, partition, Phi and Lambda as the oracle."""
    from paper_2010_10272_gb300 import HGP
    hg = synth.config_powerlaw(scale=0.002)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4, seed=2)
    want, _ = o.refine(3)
    for debug in (REORDER, KEEP):
        h = HGP.from_hypergraph(hg, subrounds=4, seed=2, debug=debug)
        np.testing.assert_array_equal(h.refine(3)[:, :5], want)
        compare_state(h, o)
        h.close()


def test_degenerate_nets():
    # empty nets, single-pin nets, isolated vertices, a vertex in every third net
    from paper_2010_10272_gb300 import HGP
    n, m = 3000, 2000
    rng = np.random.default_rng(5)
    nets = []
    for e in range(m):
        s = int(rng.integers(0, 6)) if e % 7 else int(rng.integers(40, 90))
        pins = set(rng.choice(n - 100, size=s, replace=False).tolist()) if s else set()
        if e % 3 == 0:
            pins.add(n - 101)
        nets.append(sorted(pins))
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in nets])
    pins = np.array([v for x in nets for v in x], np.int32)
    nw = rng.integers(1, 9, size=m).astype(np.int32)
    part = rng.integers(0, 4, size=n).astype(np.int32)
    for debug in (REORDER, REORDER | 2):
        h = HGP(n, m, off, pins, 4, 0.1, part, net_w=nw, subrounds=2, debug=debug)
        o = oracle.Oracle(n, m, off, pins, 4, 0.1, part, None, nw, 2, 0)
        compare_state(h, o)
        np.testing.assert_array_equal(h.refine(3)[:, :5], o.refine(3)[0])
        compare_state(h, o)


@pytest.mark.parametrize("phi_width", [0, 1, 2])
def test_large_net_prefix(phi_width):
    """Nets of 256 pins and more come first in internal order and get their own CTAs at
    creation and initialisation (pair scatter in 8192-pin chunks): nets of exactly 256 and 257
    pins (chunk edges on and off net edges), nets longer than a chunk, wide-tier nets."""
    from paper_2010_10272_gb300 import HGP
    rng = np.random.default_rng(11)
    n = 30000
    sizes = [256] * 70 + [257] * 40 + [300, 1000, 8192, 9000, 20000, 12000] + [255] * 5
    sizes += rng.integers(0, 9, size=2500).tolist()
    sizes = rng.permutation(np.array(sizes, np.int64))
    nets = [np.sort(rng.choice(n, size=int(sz), replace=False)) for sz in sizes]
    m = len(nets)
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    pins = np.concatenate(nets).astype(np.int32)
    nw = rng.integers(1, 5, size=m).astype(np.int32)
    part = rng.integers(0, 6, size=n).astype(np.int32)
    for debug in (REORDER, REORDER | 2):
        h = HGP(n, m, off, pins, 6, 0.05, part, net_w=nw, subrounds=3, phi_width=phi_width, debug=debug | 1)
        o = oracle.Oracle(n, m, off, pins, 6, 0.05, part, None, nw, 3, 0)
        compare_state(h, o)
        np.testing.assert_array_equal(h.refine(3)[:, :5], o.refine(3)[0])
        compare_state(h, o)
        h.set_partition(part)                       # initialisation again, from the start partition
        o2 = oracle.Oracle(n, m, off, pins, 6, 0.05, part, None, nw, 3, 0)
        compare_state(h, o2)
        h.close()


@pytest.mark.parametrize("balance,revert", [(True, False), (False, True), (True, True)])
def test_variants_reordered(balance, revert):
    from paper_2010_10272_gb300 import HGP
    hg = synth.random_small(61, 12000, 11000, 8, max_size=40, weighted=True, rounds=4)
    kw = dict(balance_moves=balance, revert_negative=revert)
    h = HGP.from_hypergraph(hg, subrounds=3, seed=5, debug=REORDER, **kw)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=3, seed=5, **kw)
    got = h.refine(4)
    want, _ = o.refine(4)
    np.testing.assert_array_equal(got[:, :5], want)
    np.testing.assert_array_equal(got[:, 6], o.reverted)
    compare_state(h, o)


def test_rebalance_and_exact_gains_reordered():
    from paper_2010_10272_gb300 import HGP
    hg = synth.random_small(62, 9000, 8000, 16, max_size=30, weighted=True, eps=0.05)
    part = hg.part.copy()
    part[:4000] = 0
    h = HGP.from_hypergraph(hg, part=part, subrounds=2, seed=1, debug=REORDER)
    o = oracle.Oracle.from_hypergraph(hg, part=part, subrounds=2, seed=1)
    st, ph = h.rebalance(12)
    want, want_ph, _ = o.rebalance(12, log_moves=True)
    np.testing.assert_array_equal(ph, want_ph)
    np.testing.assert_array_equal(st[:, :5], want)
    compare_state(h, o)
    rng = np.random.default_rng(3)
    cur = o.partition()
    verts = rng.permutation(hg.n)[:3000]
    to = rng.integers(0, 15, size=verts.size)
    a = cur[verts]
    to = np.where(to >= a, to + 1, to)
    moves = np.stack([verts, a, to], axis=1).astype(np.int32)
    np.testing.assert_array_equal(h.exact_gains(moves), o.exact_gains(moves))


def test_checkpoint_across_layouts():
    """A checkpoint names nets in input order, so it resumes in either layout."""
    from paper_2010_10272_gb300 import HGP
    hg = synth.random_small(63, 15000, 14000, 32, max_size=20, weighted=True, rounds=5)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=3, seed=4)
    want, _ = o.refine(5)
    for src, dst in ((REORDER, KEEP), (KEEP, REORDER)):
        a = HGP.from_hypergraph(hg, subrounds=3, seed=4, debug=src)
        first = a.refine(2)[:, :5]
        st = a.export_state()
        b = HGP.from_hypergraph(hg, subrounds=3, seed=4, debug=dst)
        b.import_state(st)
        rest = b.refine(3)[:, :5]
        np.testing.assert_array_equal(np.concatenate([first, rest]), want)
        np.testing.assert_array_equal(b.partition(), o.partition())
        b.close()
        a.close()


def test_batch_of_mixed_layouts():
    from paper_2010_10272_gb300 import HGP, Batch
    members = [synth.random_small(700 + i, 3000 + 1000 * i, 2800 + 900 * i, k, max_size=25, weighted=True, rounds=3)
               for i, k in enumerate((4, 33, 64, 16))]
    hs = [HGP.from_hypergraph(hg, subrounds=3, seed=2, debug=(REORDER if i % 2 == 0 else KEEP))
          for i, hg in enumerate(members)]
    got = Batch(hs).refine(3)
    for i, hg in enumerate(members):
        o = oracle.Oracle.from_hypergraph(hg, subrounds=3, seed=2)
        want, _ = o.refine(3)
        np.testing.assert_array_equal(got[i, :, :5], want)
        compare_state(hs[i], o)
