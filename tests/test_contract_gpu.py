"""GPU parity of contraction (Sec. 3.2) against the oracle: coarse sizes, offsets, pins,
vertex and net weights and the vertex map, bit-exact; projection and a two-level hierarchy."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_10272_gb300 import build as b
    b.build()
    oracle.build()


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _both(hg, cluster):
    from paper_2010_10272_gb300 import Coarse
    c = Coarse(hg.n, hg.m, _dev(hg.net_off), _dev(hg.pins), _dev(hg.vertex_w), _dev(hg.net_w),
               _dev(cluster.astype(np.int32)))
    got = c.to_host()
    want = oracle.contract(hg.n, hg.m, hg.net_off, hg.pins, hg.vertex_w, hg.net_w, cluster)
    assert (got["n"], got["m"]) == (want["n"], want["m"])
    for key in ("net_off", "pins", "vertex_w", "net_w", "map"):
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)
    return c, got


def _pairs(n, seed):
    """Seeded clustering of about n/2 clusters: a permutation cut into consecutive pairs."""
    perm = np.random.default_rng(seed).permutation(n)
    cl = np.empty(n, np.int64)
    cl[perm] = perm[(np.arange(n) // 2) * 2]
    return cl


@pytest.mark.parametrize("seed,n,m,max_size,weighted,factor", [
    (1, 5000, 4000, 6, False, 2), (2, 7001, 6000, 12, True, 3), (3, 3000, 5000, 40, True, 5),
    (4, 2049, 2500, 300, True, 2), (5, 9999, 8000, 3, False, 10), (6, 4000, 3000, 90, False, 50)])
def test_random_clusterings(seed, n, m, max_size, weighted, factor):
    hg = synth.random_small(400 + seed, n, m, 4, max_size=max_size, weighted=weighted)
    rng = np.random.default_rng(seed)
    cluster = rng.integers(0, max(1, n // factor), size=n)
    _both(hg, cluster)


def test_pairs_and_identity_and_single():
    hg = synth.random_small(411, 6000, 5000, 8, max_size=9, weighted=True)
    _both(hg, _pairs(hg.n, 1))
    _both(hg, np.arange(hg.n))
    _, one = _both(hg, np.full(hg.n, 17))
    assert one["n"] == 1 and one["m"] == 0


def test_many_identical_nets():
    # many nets collapse onto few pin sets: identical-net merging with large groups
    rng = np.random.default_rng(7)
    hg = synth.random_small(412, 4000, 20000, 4, max_size=5, weighted=True)
    _both(hg, rng.integers(0, 40, size=hg.n))


def test_powerlaw_scaled_with_large_nets():
    hg = synth.config_powerlaw(scale=0.004)            # nets up to thousands of pins
    _both(hg, _pairs(hg.n, 2))


def test_projection_and_hierarchy():
    """Two levels: contract, refine the coarse level on the GPU, project, and check that the
    fine objective equals the coarse one (contraction preserves (lambda-1) under projection)."""
    from paper_2010_10272_gb300 import HGP
    hg = synth.random_small(413, 20000, 18000, 8, max_size=8, weighted=True, eps=0.05)
    c, got = _both(hg, _pairs(hg.n, 3))
    cpart = torch.from_numpy(hg.part[np.unique(got["map"], return_index=True)[1]].astype(np.int32)).cuda()
    hc = c.handle(hg.k, hg.eps, cpart, subrounds=4)
    hc.refine(3)
    refined = torch.from_numpy(hc.partition()).cuda()
    fine = torch.empty(hg.n, dtype=torch.int32, device="cuda")
    c.project(refined, fine)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fine.cpu().numpy(), hc.partition()[got["map"]])
    hf = HGP.from_hypergraph(hg, part=fine.cpu().numpy())
    assert hf.objective() == hc.objective()
    # a second level from the first level's arrays
    a = c.device_arrays()
    from paper_2010_10272_gb300 import Coarse
    c2 = Coarse(c.n, c.m, a["net_off"], a["pins"], a["vertex_w"], a["net_w"],
                _dev(_pairs(c.n, 4).astype(np.int32)))
    h1 = c.to_host()
    want2 = oracle.contract(h1["n"], h1["m"], h1["net_off"], h1["pins"], h1["vertex_w"], h1["net_w"],
                            _pairs(c.n, 4))
    got2 = c2.to_host()
    for key in ("net_off", "pins", "vertex_w", "net_w", "map"):
        np.testing.assert_array_equal(got2[key], want2[key], err_msg=key)


def test_invalid_cluster_ids():
    from paper_2010_10272_gb300 import Coarse, HGPError
    hg = synth.random_small(414, 100, 80, 2)
    bad = np.zeros(hg.n, np.int32)
    bad[5] = hg.n
    with pytest.raises(HGPError):
        Coarse(hg.n, hg.m, _dev(hg.net_off), _dev(hg.pins), None, None, _dev(bad))


def test_all_levels_of_one_hierarchy_in_one_batch():
    """Levels H0..H3 from repeated contraction, refined together in one batch (one launch per
    phase over all levels): every level's result equals the level refined alone, and the
    oracle's on the coarse arrays."""
    from paper_2010_10272_gb300 import HGP, Batch, Coarse
    hg = synth.random_small(420, 30000, 26000, 8, max_size=8, weighted=True, eps=0.05)
    levels = [hg]
    coarse = []
    cur = {"n": hg.n, "m": hg.m, "net_off": hg.net_off, "pins": hg.pins,
           "vertex_w": hg.vertex_w, "net_w": hg.net_w}
    for lv in range(3):
        c = Coarse(cur["n"], cur["m"], _dev(cur["net_off"]), _dev(cur["pins"]), _dev(cur["vertex_w"]),
                   _dev(cur["net_w"]), _dev(_pairs(cur["n"], 10 + lv).astype(np.int32)))
        coarse.append(c)
        cur = c.to_host()
    arrays = [{"n": hg.n, "m": hg.m, "net_off": hg.net_off, "pins": hg.pins, "vertex_w": hg.vertex_w,
               "net_w": hg.net_w}] + [c.to_host() for c in coarse]
    rng = np.random.default_rng(5)
    parts = [rng.integers(0, hg.k, size=a["n"]).astype(np.int32) for a in arrays]

    def make(i):
        a = arrays[i]
        return HGP(a["n"], a["m"], a["net_off"], a["pins"], hg.k, hg.eps, parts[i], a["vertex_w"], a["net_w"],
                   subrounds=3, seed=i)
    hs = [make(i) for i in range(len(arrays))]
    b = Batch(hs)
    got = b.refine(4)
    for i, a in enumerate(arrays):
        alone = make(i)
        np.testing.assert_array_equal(got[i][:, :5], alone.refine(4)[:, :5])
        np.testing.assert_array_equal(hs[i].partition(), alone.partition())
        o = oracle.Oracle(a["n"], a["m"], a["net_off"], a["pins"], hg.k, hg.eps, parts[i], a["vertex_w"],
                          a["net_w"], 3, i)
        np.testing.assert_array_equal(got[i][:, :5], o.refine(4)[0])
    b.close()
    assert arrays[-1]["n"] < arrays[0]["n"] // 6
