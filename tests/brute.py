"""Brute-force statements of the paper's definitions, for pinning the oracle on tiny inputs.

Nothing here calls the oracle or the CUDA library.  Every quantity is computed from its
definition in the most direct way available:

* the objective (lambda-1)(Pi) from connectivity sets built as Python sets (Sec. 2);
* the gain of a move as the objective reduction it causes, obj(Pi) - obj(Pi[u->i])
  (the sentence after the objective's definition in Sec. 2), not through b(u) - p_i(u);
* eligibility as "u or a vertex sharing a net with u was moved in the previous round"
  (Sec. 6), from the set of moved vertices rather than from per-net flags;
* the sub-round hash from the published SplitMix64 output function.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np

M64 = (1 << 64) - 1


def splitmix64_output(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def subround(seed: int, rnd: int, u: int, S: int) -> int:
    return splitmix64_output(seed ^ ((rnd << 32) | u)) % S


class Tiny:
    """A hypergraph held as Python lists, for brute force."""

    def __init__(self, n, nets: Sequence[Sequence[int]], k, eps, vw=None, nw=None):
        self.n, self.k, self.eps = n, k, eps
        self.nets = [sorted(set(int(v) for v in e)) for e in nets]
        self.m = len(self.nets)
        self.vw = [1] * n if vw is None else [int(x) for x in vw]
        self.nw = [1] * self.m if nw is None else [int(x) for x in nw]
        self.inc: List[List[int]] = [[] for _ in range(n)]
        for e, pins in enumerate(self.nets):
            for v in pins:
                self.inc[v].append(e)

    @classmethod
    def from_hypergraph(cls, hg):
        nets = [hg.pins[hg.net_off[e]:hg.net_off[e + 1]].tolist() for e in range(hg.m)]
        return cls(hg.n, nets, hg.k, hg.eps,
                   None if hg.vertex_w is None else hg.vertex_w.tolist(),
                   None if hg.net_w is None else hg.net_w.tolist())

    def csr(self):
        off = np.zeros(self.m + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(e) for e in self.nets])
        pins = np.array([v for e in self.nets for v in e], dtype=np.int32)
        return off, pins

    # Sec. 2: L_max = (1+eps) * ceil(c(V)/k), rounded down to an integer weight
    def lmax(self) -> int:
        total = sum(self.vw)
        avg = -(-total // self.k)
        return int(np.floor((1.0 + self.eps) * avg))

    def objective(self, part) -> int:
        """(lambda-1)(Pi) = sum_e (|{Pi(v) : v in e}| - 1) * omega(e); empty nets count 0."""
        total = 0
        for e, pins in enumerate(self.nets):
            blocks = {int(part[v]) for v in pins}
            if blocks:
                total += (len(blocks) - 1) * self.nw[e]
        return total

    def gain(self, part, u: int, i: int) -> int:
        """Objective reduction of moving u to block i."""
        moved = list(part)
        moved[u] = i
        return self.objective(part) - self.objective(moved)

    def block_weights(self, part) -> List[int]:
        w = [0] * self.k
        for v in range(self.n):
            w[int(part[v])] += self.vw[v]
        return w

    def phi(self, part) -> np.ndarray:
        out = np.zeros((self.m, self.k), dtype=np.int64)
        for e, pins in enumerate(self.nets):
            for v in pins:
                out[e, int(part[v])] += 1
        return out

    def neighbours(self, u: int):
        out = set()
        for e in self.inc[u]:
            out.update(self.nets[e])
        return out


def eligible_after(t: Tiny, moved_prev: Optional[set]) -> set:
    """Eligible vertices of a round (Sec. 6): every vertex in the first round (moved_prev is
    None), otherwise the vertices that share a net with a vertex moved in the round before
    (a moved vertex with at least one net is its own neighbour)."""
    if moved_prev is None:
        return set(range(t.n))
    elig = set()
    for v in moved_prev:
        if t.inc[v]:
            elig |= t.neighbours(v)
    return elig


def candidates(t: Tiny, part, elig, r: int, s: int, S: int, seed: int = 0,
               balance_moves: bool = False) -> Dict[int, tuple]:
    """{u: (target, gain)} of sub-round s of round r: every eligible vertex active in s picks
    the block with the largest objective reduction among those with room for it (block
    weights of `part`), smallest block on ties, if that reduction is positive."""
    lmax = t.lmax()
    w = t.block_weights(part)
    cands: Dict[int, tuple] = {}
    for u in sorted(elig):
        if subround(seed, r, u, S) != s:
            continue
        best = None
        for i in range(t.k):
            if i == part[u]:
                continue
            g = t.gain(part, u, i)
            if g > 0 and w[i] + t.vw[u] <= lmax and (best is None or g > best[1]):
                best = (i, g)
        if best is None and balance_moves:
            # a zero-gain move to a block it leaves more balanced than a: lightest first
            zs = [i for i in range(t.k) if i != part[u] and t.gain(part, u, i) == 0
                  and w[i] + t.vw[u] <= lmax and w[i] + t.vw[u] < w[part[u]]]
            if zs:
                best = (min(zs, key=lambda i: (w[i], i)), 0)
        if best is not None:
            cands[u] = best
    return cands


def lp_rounds(t: Tiny, part, rounds: int, S: int = 4, seed: int = 0, start_round: int = 0,
              moved_prev: Optional[set] = None, balance_moves: bool = False,
              revert_negative: bool = False, reverted: Optional[list] = None):
    """Synchronous LP rounds with definitional gains.  Returns (part, per-round stats,
    move log [(global sub-round, u, from, to)], moved set of the last round).

    Stats per round: (objective, candidates, approved, eligible, max block weight).
    revert_negative: each approved move is performed in ascending vertex id and its
    attributed gain is the objective it removes at that moment; after the sub-round the moves
    with a negative one go back (logged as reverse moves); per-round counts go to `reverted`."""
    part = [int(x) for x in part]
    lmax = t.lmax()
    stats, log = [], []
    all_elig = moved_prev is None
    for rr in range(rounds):
        r = start_round + rr
        elig = eligible_after(t, None if all_elig else moved_prev)
        moved_now = set()
        n_cand = n_appr = n_rev = 0
        for s in range(S):
            w = t.block_weights(part)
            cands = candidates(t, part, elig, r, s, S, seed, balance_moves)
            n_cand += len(cands)
            approved = []
            for blk in range(t.k):
                lst = sorted((u for u in cands if cands[u][0] == blk),
                             key=lambda u: (-cands[u][1], u))
                acc = 0
                for u in lst:
                    acc += t.vw[u]
                    if w[blk] + acc <= lmax:
                        approved.append(u)
            attr = {}
            for u in sorted(approved):
                log.append((r * S + s, u, part[u], cands[u][0]))
                attr[u] = (t.gain(part, u, cands[u][0]), part[u])
                part[u] = cands[u][0]
                moved_now.add(u)
            n_appr += len(approved)
            if revert_negative:
                for u in sorted(approved):
                    if attr[u][0] < 0:
                        log.append((r * S + s, u, part[u], attr[u][1]))
                        part[u] = attr[u][1]
                        n_rev += 1
        stats.append((t.objective(part), n_cand, n_appr, len(elig), max(t.block_weights(part))))
        if reverted is not None:
            reverted.append(n_rev)
        moved_prev = moved_now
        all_elig = False
    return part, stats, log, moved_prev


def random_tiny(rng: np.random.Generator, n: int, m: int, k: int, max_size: int = 4,
                weighted: bool = False, eps: float = 0.2) -> Tiny:
    nets = []
    for _ in range(m):
        s = int(rng.integers(1, max_size + 1))
        nets.append(rng.choice(n, size=min(s, n), replace=False).tolist())
    vw = rng.integers(1, 4, size=n).tolist() if weighted else None
    nw = rng.integers(1, 6, size=m).tolist() if weighted else None
    return Tiny(n, nets, k, eps, vw, nw)


def rebalance(t: Tiny, part, max_passes: int, S: int = 4, seed: int = 0):
    """Rebalancing passes (Sec. 8) with definitional gains (objective differences).
    Returns (part, per-pass stats (objective, candidates, approved, considered, max block
    weight), phases, move log [(pass * S + sub-round, u, from, to)])."""
    part = [int(x) for x in part]
    lmax = t.lmax()
    stats, phases, log = [], [], []
    phase, p = 1, 0
    while p < max_passes and max(t.block_weights(part)) > lmax:
        n_cand = n_appr = n_cons = 0
        for s in range(S):
            w = t.block_weights(part)
            cands = {}
            for u in range(t.n):
                a = part[u]
                if subround(seed, (1 << 30) + p, u, S) != s or w[a] <= lmax:
                    continue
                n_cons += 1
                room = [i for i in range(t.k) if i != a and w[i] + t.vw[u] <= lmax]
                if not room:
                    continue
                best = max(room, key=lambda i: (t.gain(part, u, i), -i))
                g = t.gain(part, u, best)
                if phase == 1 and g < 0:
                    continue
                cands[u] = (best, g)
            n_cand += len(cands)
            order = sorted(cands, key=lambda u: (-cands[u][1], u))
            selected = set()
            for a in range(t.k):
                left = 0
                for u in order:
                    if part[u] != a:
                        continue
                    if left < w[a] - lmax:
                        selected.add(u)
                    left += t.vw[u]
            approved = []
            for blk in range(t.k):
                acc = 0
                for u in order:
                    if u in selected and cands[u][0] == blk:
                        acc += t.vw[u]
                        if w[blk] + acc <= lmax:
                            approved.append(u)
            for u in sorted(approved):
                log.append((p * S + s, u, part[u], cands[u][0]))
                part[u] = cands[u][0]
            n_appr += len(approved)
        stats.append((t.objective(part), n_cand, n_appr, n_cons, max(t.block_weights(part))))
        phases.append(phase)
        p += 1
        if phase == 1:
            phase = 2
        elif n_appr == 0:
            break
    return part, stats, phases, log
