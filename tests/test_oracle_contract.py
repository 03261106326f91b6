"""Pins for the oracle's contraction (Sec. 3.2): a hand-derived example, a brute-force
construction from the definition, and the property that makes contraction correct: every
coarse partition has the same connectivity objective as its projection to the fine vertices."""
import numpy as np
import pytest

import oracle
from brute import Tiny, random_tiny


def _contract(t: Tiny, cluster):
    off, pins = t.csr()
    return oracle.contract(t.n, t.m, off, pins, np.array(t.vw, np.int32), np.array(t.nw, np.int32),
                           np.array(cluster, np.int32))


def brute_contract(t: Tiny, cluster):
    """The definition with Python sets and dicts."""
    used = sorted(set(int(c) for c in cluster))
    cid = {c: i for i, c in enumerate(used)}
    vmap = [cid[int(c)] for c in cluster]
    vw = [0] * len(used)
    for u in range(t.n):
        vw[vmap[u]] += t.vw[u]
    groups = {}                   # pin tuple -> [smallest original net id, weight]
    for e, net in enumerate(t.nets):
        key = tuple(sorted(set(vmap[v] for v in net)))
        if len(key) < 2:
            continue
        if key in groups:
            groups[key][1] += t.nw[e]
        else:
            groups[key] = [e, t.nw[e]]
    nets = sorted(groups.items(), key=lambda kv: kv[1][0])
    return vmap, vw, [list(k) for k, _ in nets], [w for _, (_, w) in nets]


def test_hand_example():
    # 6 vertices, clusters {0,1} -> id 3, {2} -> 5, {3,4,5} -> 0 (ids 3, 5, 0 remap to 1, 2, 0).
    # Nets: {0,1} (w 2) becomes {1}: removed; {1,2} (w 3) -> {1,2}; {0,2,3} (w 1) -> {0,1,2};
    # {3,4} (w 7) -> {0}: removed; {2,5} (w 4) -> {0,2}; {0,5} (w 5) -> {0,1};
    # {1,2,4} (w 6) -> {0,1,2}: identical to net 2, weights 1 + 6 = 7 at net 2's position.
    t = Tiny(6, [[0, 1], [1, 2], [0, 2, 3], [3, 4], [2, 5], [0, 5], [1, 2, 4]], 2, 0.1,
             vw=[1, 2, 3, 4, 5, 6], nw=[2, 3, 1, 7, 4, 5, 6])
    c = _contract(t, [3, 3, 5, 0, 0, 0])
    assert c["n"] == 3 and c["map"].tolist() == [1, 1, 2, 0, 0, 0]
    assert c["vertex_w"].tolist() == [15, 3, 3]
    assert c["m"] == 4
    assert c["net_off"].tolist() == [0, 2, 5, 7, 9]
    assert c["pins"].tolist() == [1, 2, 0, 1, 2, 0, 2, 0, 1]
    assert c["net_w"].tolist() == [3, 7, 4, 5]


@pytest.mark.parametrize("seed", range(12))
def test_matches_bruteforce(seed):
    rng = np.random.default_rng(1500 + seed)
    n = int(rng.integers(5, 30))
    t = random_tiny(rng, n, int(rng.integers(1, 40)), 2, max_size=6, weighted=True)
    cluster = rng.integers(0, max(1, n // int(rng.integers(1, 4))), size=n)
    c = _contract(t, cluster)
    vmap, vw, nets, nw = brute_contract(t, cluster)
    assert c["map"].tolist() == vmap
    assert c["vertex_w"].tolist() == vw
    assert c["m"] == len(nets)
    got = [c["pins"][c["net_off"][i]:c["net_off"][i + 1]].tolist() for i in range(c["m"])]
    assert got == nets
    assert c["net_w"].tolist() == nw


@pytest.mark.parametrize("seed", range(8))
def test_objective_preserved_under_projection(seed):
    # (lambda-1) of a coarse partition equals (lambda-1) of its projection: removed single-pin
    # nets are never cut, and merged identical nets are cut together with summed weight
    rng = np.random.default_rng(1600 + seed)
    n, k = 40, int(rng.integers(2, 6))
    t = random_tiny(rng, n, 60, k, max_size=7, weighted=True)
    cluster = rng.integers(0, n // 3, size=n)
    c = _contract(t, cluster)
    coarse = Tiny(c["n"], [c["pins"][c["net_off"][i]:c["net_off"][i + 1]].tolist() for i in range(c["m"])],
                  k, 0.1, c["vertex_w"].tolist(), c["net_w"].tolist())
    for _ in range(5):
        cp = rng.integers(0, k, size=c["n"])
        fine = cp[c["map"]]
        assert coarse.objective(cp) == t.objective(fine)
        assert coarse.block_weights(cp) == t.block_weights(fine)


def test_identity_and_single_cluster():
    rng = np.random.default_rng(3)
    t = random_tiny(rng, 20, 30, 2, max_size=5, weighted=True)
    c = _contract(t, np.arange(20))
    vmap, vw, nets, nw = brute_contract(t, np.arange(20))
    assert c["map"].tolist() == list(range(20)) and c["vertex_w"].tolist() == t.vw
    assert c["m"] == len(nets)
    one = _contract(t, np.full(20, 7))
    assert one["n"] == 1 and one["m"] == 0 and one["vertex_w"].tolist() == [sum(t.vw)]


def test_rejects_bad_cluster_ids():
    t = Tiny(3, [[0, 1, 2]], 2, 0.1)
    with pytest.raises(ValueError):
        _contract(t, [0, 3, 1])
