"""Full-size GPU checks in the launch configuration bench.py times (device-resident inputs,
hgp_create_device, default options, hgp_refine over the workload's rounds), element by element
against the oracle.

* row-net workload (2*10^6 x 2*10^6, k=8, 10 rounds).
* power-law workload (n = m = 5*10^7, P = 3.45*10^8, k=64, 5 rounds): every round's statistics,
  the final partition, block weights, objective, Lambda of every net and the whole Phi table
  (compared in row blocks), plus the round-0 candidates of sampled vertices against the oracle's
  sample routine.  The oracle runs its independent loops on all host cores (identical results
  for any thread count) so that the five rounds take minutes, not an hour.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


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


def _lambda_from_phi_rows(rows):
    bits = np.zeros(rows.shape[0], dtype=np.uint64)
    for i in range(rows.shape[1]):
        bits |= (rows[:, i] > 0).astype(np.uint64) << np.uint64(i)
    return bits


def _objective(hg, lam):
    lam_count = np.bitwise_count(lam).astype(np.int64)
    w = np.ones(hg.m, np.int64) if hg.net_w is None else hg.net_w.astype(np.int64)
    return int((np.maximum(lam_count - 1, 0) * w).sum())


def test_rownet_full_parity():
    hg = synth.config_rownet()
    h = _device_handle(hg)
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4, threads=THREADS)
    assert h.info()["lmax"] == o.lmax == 257_500
    got = h.refine(hg.rounds)[:, :5]
    want, _ = o.refine(hg.rounds)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(h.partition(), o.partition())
    np.testing.assert_array_equal(h.block_weights(), o.block_weights())
    np.testing.assert_array_equal(h.phi(), o.phi())
    assert h.objective() == o.objective() == h.objective_from_phi()


def test_powerlaw_full_oracle_parity():
    hg = synth.config_powerlaw()
    assert hg.n == 50_000_000 and hg.k == 64
    h = _device_handle(hg)
    info = h.info()
    assert info["lmax"] == 804_687 and info["phi_width"] == 2 and info["wide_nets"] > 0
    # round 0, sub-round 0: sampled candidates against the oracle's sample routine
    rng = np.random.default_rng(2024)
    sample = np.sort(rng.choice(hg.n, size=20_000, replace=False)).astype(np.int32)
    want_t, want_g = oracle.sample_candidates(hg, sample, s=0, subrounds=4, seed=0)
    t, g = h.debug_candidates(0)
    np.testing.assert_array_equal(t[sample], want_t)
    np.testing.assert_array_equal(g[sample], want_g)
    assert (want_t >= 0).sum() > 1000
    del t, g
    lam0 = _lambda_from_partition(hg, hg.part)
    np.testing.assert_array_equal(h.lam(), lam0)
    obj0 = h.objective()
    assert obj0 == _objective(hg, lam0)
    # every round on the GPU, then the whole state read back; the handle is freed before the
    # oracle is built (host memory)
    got = h.refine(hg.rounds)
    part, bw, lam = h.partition(), h.block_weights(), h.lam()
    obj, obj_phi = h.objective(), h.objective_from_phi()
    phi = h.phi().reshape(hg.m, hg.k)
    h.close()
    del h
    torch.cuda.empty_cache()
    o = oracle.Oracle.from_hypergraph(hg, subrounds=4, threads=THREADS)
    assert o.lmax == info["lmax"] and o.objective() == obj0
    want, _ = o.refine(hg.rounds)
    np.testing.assert_array_equal(got[:, :5], want)
    np.testing.assert_array_equal(part, o.partition())
    np.testing.assert_array_equal(bw, o.block_weights())
    assert obj == obj_phi == o.objective() == want[-1, 0]
    step = 1 << 22
    for e0 in range(0, hg.m, step):
        e1 = min(hg.m, e0 + step)
        rows = o.phi_rows(e0, e1)
        if not np.array_equal(phi[e0:e1], rows):
            bad = e0 + int(np.flatnonzero((phi[e0:e1] != rows).any(axis=1))[0])
            raise AssertionError(f"Phi row of net {bad} differs: {phi[bad]} vs {rows[bad - e0]}")
        np.testing.assert_array_equal(lam[e0:e1], _lambda_from_phi_rows(rows))
    assert want[0, 3] == hg.n                       # every vertex eligible in the first round
    assert want[-1, 0] < want[0, 0] < obj0
    o.close()
