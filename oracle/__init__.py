"""CPU oracle for synchronous LP refinement under the (lambda-1) metric.

TEST INFRASTRUCTURE ONLY: the plain sequential statement of what the CUDA path computes.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``hgp_oracle.c`` (definitions of Sec. 2, gain of Sec. 5, label
propagation of Sec. 6 in the synchronous sub-round form); this module only builds it with
gcc and marshals arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STAT_FIELDS = ("objective", "candidates", "approved", "eligible", "max_block_weight")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, portable flags).

    ``HGP_ORACLE_LIB`` names an already built oracle library to use instead (the mutation
    tests point it at deliberately broken copies)."""
    if os.environ.get("HGP_ORACLE_LIB"):
        return os.environ["HGP_ORACLE_LIB"]
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        lib.oracle_create.restype = P
        lib.oracle_create.argtypes = [i32, i32, P, P, P, P, i32, f64, P, i32, u64]
        lib.oracle_destroy.argtypes = [P]
        lib.oracle_refine.restype = ctypes.c_int
        lib.oracle_refine.argtypes = [P, i32, P, P, i64, P]
        lib.oracle_gain.restype = i64
        lib.oracle_gain.argtypes = [P, i32, i32]
        lib.oracle_candidates.argtypes = [P, i32, P, P]
        lib.oracle_objective.restype = i64
        lib.oracle_objective.argtypes = [P]
        lib.oracle_lmax_of.restype = i64
        lib.oracle_lmax_of.argtypes = [P]
        lib.oracle_round_of.restype = i64
        lib.oracle_round_of.argtypes = [P]
        lib.oracle_lmax.restype = i64
        lib.oracle_lmax.argtypes = [i64, i32, f64]
        lib.oracle_mix64.restype = u64
        lib.oracle_mix64.argtypes = [u64]
        lib.oracle_subround_of.restype = i32
        lib.oracle_subround_of.argtypes = [u64, i64, i32, i32]
        for name in ("oracle_get_partition", "oracle_get_block_weights", "oracle_get_phi"):
            getattr(lib, name).argtypes = [P, P]
        lib.oracle_set_variant.argtypes = [P, i32, i32]
        lib.oracle_set_threads.argtypes = [P, i32]
        lib.oracle_get_phi_rows.argtypes = [P, i32, i32, P]
        lib.oracle_contract.restype = ctypes.c_int
        lib.oracle_contract.argtypes = [i32, i32, P, P, P, P, P, ctypes.POINTER(P)]
        lib.oracle_coarse_destroy.argtypes = [P]
        lib.oracle_coarse_sizes.argtypes = [P, P, P, P]
        lib.oracle_coarse_copy.argtypes = [P, P, P, P, P, P]
        lib.oracle_rebalance.restype = ctypes.c_int
        lib.oracle_rebalance.argtypes = [P, i32, P, P, P, P, i64, P]
        lib.oracle_exact_gains.restype = ctypes.c_int
        lib.oracle_exact_gains.argtypes = [P, i32, P, P]
        lib.oracle_sample_candidates.restype = ctypes.c_int
        lib.oracle_sample_candidates.argtypes = [i32, i32, P, P, P, P, i32, f64, P, i32, u64,
                                                 i32, i32, P, P, P]
        _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def lmax(total_weight: int, k: int, eps: float) -> int:
    return int(_load().oracle_lmax(int(total_weight), int(k), float(eps)))


def mix64(x: int) -> int:
    return int(_load().oracle_mix64(x))


def subround_of(seed: int, rnd: int, u: int, S: int) -> int:
    return int(_load().oracle_subround_of(seed, rnd, u, S))


class Oracle:
    """Sequential oracle state for one hypergraph and partition."""

    def __init__(self, n, m, net_off, pins, k, eps, part, vertex_w=None, net_w=None,
                 subrounds: int = 4, seed: int = 0, balance_moves: bool = False,
                 revert_negative: bool = False, threads: int = 1):
        lib = _load()
        self._lib = lib
        self.n, self.m, self.k = int(n), int(m), int(k)
        self.subrounds = int(subrounds)
        self._keep = [_c(net_off, np.int64), _c(pins, np.int32), _c(vertex_w, np.int32),
                      _c(net_w, np.int32), _c(part, np.int32)]
        off, pn, vw, nw, pt = self._keep
        self._h = lib.oracle_create(self.n, self.m, _ptr(off), _ptr(pn), _ptr(vw), _ptr(nw),
                                    self.k, float(eps), _ptr(pt), self.subrounds, int(seed))
        if not self._h:
            raise ValueError("oracle_create rejected the input")
        self._keep = None
        lib.oracle_set_variant(self._h, int(bool(balance_moves)), int(bool(revert_negative)))
        lib.oracle_set_threads(self._h, int(threads))

    @classmethod
    def from_hypergraph(cls, hg, subrounds: int = 4, seed: int = 0, part=None, **variant):
        return cls(hg.n, hg.m, hg.net_off, hg.pins, hg.k, hg.eps,
                   hg.part if part is None else part, hg.vertex_w, hg.net_w, subrounds, seed,
                   **variant)

    def close(self):
        if self._h:
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refine(self, rounds: int, log_moves: bool = False, max_moves: int = 1 << 20):
        """Runs `rounds` rounds. Returns (stats [rounds x 5] int64, moves or None); the
        per-round count of reverted moves (revert variant) is left in `self.reverted`.

        moves: int64 [count x 4] = (global sub-round index, u, from, to); a reverted move
        appears a second time, from its target back to its source, after its sub-round's
        moves."""
        stats = np.zeros((rounds, len(STAT_FIELDS) + 1), dtype=np.int64)
        moves = np.zeros((max_moves, 4), dtype=np.int64) if log_moves else None
        cnt = ctypes.c_int64(0)
        rc = self._lib.oracle_refine(self._h, int(rounds), _ptr(stats), _ptr(moves),
                                     int(max_moves if log_moves else 0), ctypes.byref(cnt))
        if rc != 0:
            raise MemoryError("oracle_refine failed")
        if log_moves:
            if cnt.value > max_moves:
                raise ValueError("move log truncated")
            moves = moves[:cnt.value].copy()
        self.reverted = stats[:, len(STAT_FIELDS)].copy()
        return stats[:, :len(STAT_FIELDS)].copy(), moves

    def rebalance(self, max_passes: int, log_moves: bool = False, max_moves: int = 1 << 20):
        """Rebalancing passes (Sec. 8).  Returns (stats [passes x 5] int64, phases [passes]
        int32, moves or None); moves as in refine, first field = pass * S + sub-round."""
        stats = np.zeros((max(1, max_passes), len(STAT_FIELDS) + 1), dtype=np.int64)
        phases = np.zeros(max(1, max_passes), dtype=np.int32)
        moves = np.zeros((max_moves, 4), dtype=np.int64) if log_moves else None
        npass = ctypes.c_int32(0)
        cnt = ctypes.c_int64(0)
        rc = self._lib.oracle_rebalance(self._h, int(max_passes), _ptr(stats), _ptr(phases),
                                        ctypes.byref(npass), _ptr(moves),
                                        int(max_moves if log_moves else 0), ctypes.byref(cnt))
        if rc != 0:
            raise MemoryError("oracle_rebalance failed")
        p = npass.value
        if log_moves:
            if cnt.value > max_moves:
                raise ValueError("move log truncated")
            moves = moves[:cnt.value].copy()
        return stats[:p, :len(STAT_FIELDS)].copy(), phases[:p].copy(), moves

    def gain(self, u: int, i: int) -> int:
        return int(self._lib.oracle_gain(self._h, int(u), int(i)))

    def candidates(self, s: int):
        t = np.zeros(self.n, dtype=np.int32)
        g = np.zeros(self.n, dtype=np.int64)
        self._lib.oracle_candidates(self._h, int(s), _ptr(t), _ptr(g))
        return t, g

    def exact_gains(self, moves) -> np.ndarray:
        """Gains of a move sequence [(u, from, to), ...] performed in order (state unchanged)."""
        mv = np.ascontiguousarray(moves, dtype=np.int32).reshape(-1, 3)
        g = np.zeros(mv.shape[0], dtype=np.int64)
        if self._lib.oracle_exact_gains(self._h, int(mv.shape[0]), _ptr(mv), _ptr(g)) != 0:
            raise ValueError("invalid move sequence")
        return g

    def objective(self) -> int:
        return int(self._lib.oracle_objective(self._h))

    @property
    def lmax(self) -> int:
        return int(self._lib.oracle_lmax_of(self._h))

    @property
    def round(self) -> int:
        return int(self._lib.oracle_round_of(self._h))

    def partition(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int32)
        self._lib.oracle_get_partition(self._h, _ptr(out))
        return out

    def block_weights(self) -> np.ndarray:
        out = np.zeros(self.k, dtype=np.int64)
        self._lib.oracle_get_block_weights(self._h, _ptr(out))
        return out

    def phi(self) -> np.ndarray:
        out = np.zeros((self.m, self.k), dtype=np.int64)
        self._lib.oracle_get_phi(self._h, _ptr(out))
        return out

    def phi_rows(self, e0: int, e1: int) -> np.ndarray:
        """Rows e0 <= e < e1 of Phi as int32 [e1 - e0, k] (for instances too large to copy whole)."""
        e0, e1 = int(e0), int(e1)
        if not 0 <= e0 <= e1 <= self.m:
            raise ValueError("row range outside [0, m]")
        out = np.zeros((e1 - e0, self.k), dtype=np.int32)
        self._lib.oracle_get_phi_rows(self._h, e0, e1, _ptr(out))
        return out


def sample_candidates(hg, sample, s: int = 0, subrounds: int = 4, seed: int = 0, part=None):
    """Round-0 candidates (target, gain) of sub-round s for the distinct vertices `sample`,
    computed from the input alone (no full Phi table)."""
    lib = _load()
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    t = np.zeros(sample.size, dtype=np.int32)
    g = np.zeros(sample.size, dtype=np.int64)
    off, pn = _c(hg.net_off, np.int64), _c(hg.pins, np.int32)
    vw, nw = _c(hg.vertex_w, np.int32), _c(hg.net_w, np.int32)
    pt = _c(hg.part if part is None else part, np.int32)
    rc = lib.oracle_sample_candidates(hg.n, hg.m, _ptr(off), _ptr(pn), _ptr(vw), _ptr(nw),
                                      hg.k, float(hg.eps), _ptr(pt), int(subrounds), int(seed),
                                      int(s), int(sample.size), _ptr(sample), _ptr(t), _ptr(g))
    if rc != 0:
        raise MemoryError("oracle_sample_candidates failed")
    return t, g


def contract(n, m, net_off, pins, vertex_w, net_w, cluster) -> dict:
    """Coarse hypergraph of a clustering (Sec. 3.2): dict with n, m, net_off int64[m+1],
    pins int32, vertex_w int64[n], net_w int64[m] and map int32[fine n]."""
    lib = _load()
    keep = [_c(net_off, np.int64), _c(pins, np.int32), _c(vertex_w, np.int32), _c(net_w, np.int32),
            _c(cluster, np.int32)]
    h = ctypes.c_void_p()
    rc = lib.oracle_contract(int(n), int(m), *[_ptr(x) for x in keep], ctypes.byref(h))
    if rc == -2:
        raise ValueError("cluster id outside [0, n)")
    if rc != 0:
        raise MemoryError("oracle_contract failed")
    try:
        n2, m2, p2 = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        lib.oracle_coarse_sizes(h, ctypes.byref(n2), ctypes.byref(m2), ctypes.byref(p2))
        out = {"n": n2.value, "m": m2.value,
               "net_off": np.zeros(m2.value + 1, np.int64), "pins": np.zeros(p2.value, np.int32),
               "vertex_w": np.zeros(n2.value, np.int64), "net_w": np.zeros(m2.value, np.int64),
               "map": np.zeros(int(n), np.int32)}
        lib.oracle_coarse_copy(h, _ptr(out["net_off"]), _ptr(out["pins"]), _ptr(out["vertex_w"]),
                               _ptr(out["net_w"]), _ptr(out["map"]))
    finally:
        lib.oracle_coarse_destroy(h)
    return out
