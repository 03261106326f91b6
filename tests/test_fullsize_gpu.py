"""Full-size GPU checks in the launch configuration bench.py times (device-resident inputs,
hgp_create_device, default options, hgp_refine over the workload's rounds).

* row-net workload (2*10^6 x 2*10^6, k=8, 10 rounds): element-by-element parity with the oracle.
* power-law workload (n = m = 5*10^7, k=64, 5 rounds): the oracle cannot hold this instance's
  Phi table, so (a) round-0 candidates of sampled vertices are compared with the oracle's
  sample routine, which counts Phi only for the nets of the sampled vertices, and (b) after all
  rounds, properties that hold at any size are checked against host recomputation from the
  returned partition: Lambda(e) of every net, the objective, block weights, balance.
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


def _device_handle(hg, S=4):
    from paper_2010_10272_gb300 import HGP
    dev = torch.device("cuda:0")
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    h = HGP(hg.n, hg.m, t(hg.net_off), t(hg.pins), hg.k, hg.eps, t(hg.part), t(hg.vertex_w),
            t(hg.net_w), subrounds=S, device=True, stream=torch.cuda.current_stream(dev))
    return h


def _lambda_from_partition(hg, part):
    """Lambda(e) as 64-bit masks: OR of (1 << Pi(v)) over the pins of each net."""
    bits = np.left_shift(np.uint64(1), part[hg.pins].astype(np.uint64))
    lam = np.zeros(hg.m, dtype=np.uint64)
    sizes = np.diff(hg.net_off)
    nz = np.flatnonzero(sizes)
    if nz.size:
        lam[nz] = np.bitwise_or.reduceat(bits, hg.net_off[:-1][nz])
    return lam


def _objective(hg, lam):
    lam_count = np.bitwise_count(lam).astype(np.int64)
    w = np.ones(hg.m, np.int64) if hg.net_w is None else hg.net_w.astype(np.int64)
    return int((np.maximum(lam_count - 1, 0) * w).sum())


def test_rownet_full_parity():
    hg = synth.config_rownet()
    h = _device_handle(hg)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4)
    assert h.info()["lmax"] == o.lmax == 257_500
    got = h.refine(hg.rounds)[:, :5]
    want, _ = o.refine(hg.rounds)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(h.partition(), o.partition())
    np.testing.assert_array_equal(h.block_weights(), o.block_weights())
    np.testing.assert_array_equal(h.phi(), o.phi())
    assert h.objective() == o.objective() == h.objective_from_phi()


def test_powerlaw_full_sampled_and_properties():
    hg = synth.config_powerlaw()
    assert hg.n == 50_000_000 and hg.k == 64
    h = _device_handle(hg)
    info = h.info()
    assert info["lmax"] == 804_687 and info["phi_width"] == 2 and info["wide_nets"] > 0
    # (a) round 0, sub-round 0: sampled candidates against the oracle's sample routine
    rng = np.random.default_rng(2024)
    sample = np.sort(rng.choice(hg.n, size=20_000, replace=False)).astype(np.int32)
    want_t, want_g = oracle.sample_candidates(hg, sample, s=0, subrounds=4, seed=0)
    t, g = h.debug_candidates(0)
    np.testing.assert_array_equal(t[sample], want_t)
    np.testing.assert_array_equal(g[sample], want_g)
    assert (want_t >= 0).sum() > 1000
    # initial state against host recomputation
    lam0 = _lambda_from_partition(hg, hg.part)
    np.testing.assert_array_equal(h.lam(), lam0)
    assert h.objective() == _objective(hg, lam0)
    # (b) all rounds, then properties of the result
    w0 = h.block_weights()
    stats = h.refine(hg.rounds)
    part = h.partition()
    assert part.min() >= 0 and part.max() < hg.k
    lam = _lambda_from_partition(hg, part)
    np.testing.assert_array_equal(h.lam(), lam)
    obj = _objective(hg, lam)
    assert h.objective() == obj == h.objective_from_phi() == stats[-1, 0]
    w = np.bincount(part, minlength=hg.k).astype(np.int64)
    np.testing.assert_array_equal(h.block_weights(), w)
    assert w.sum() == hg.n
    assert np.all(w <= np.maximum(w0, info["lmax"]))
    assert stats[0, 3] == hg.n                      # every vertex eligible in the first round
    assert np.all(stats[:, 2] <= stats[:, 1])       # approved <= candidates
    assert stats[-1, 0] < stats[0, 0] < _objective(hg, lam0)
