"""ctypes binding of libhgp (include/hgp.h).  Argument marshalling only.

Host arrays are numpy arrays; device arrays are torch CUDA tensors (their data pointers are
passed through).  Streams are torch streams or raw cudaStream_t integers.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libhgp.so")
_lock = threading.Lock()
_lib = None

STAT_FIELDS = ("objective", "candidates", "approved", "eligible", "max_block_weight", "moved_pins",
               "reverted")
PHASES = ("sublists", "gain", "approval", "apply", "round_end", "revert")

HGP_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "UNSUPPORTED", 4: "CUDA", 5: "TIMEOUT",
                6: "INTERNAL"}


class HGPError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)} ({strerror(code)})")


class Options(ctypes.Structure):
    _fields_ = [("subrounds", ctypes.c_int32), ("phi_width", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("debug", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("balance_moves", ctypes.c_int32),
                ("revert_negative", ctypes.c_int32), ("gain_ctas_per_sm", ctypes.c_int32),
                ("apply_ctas_per_sm", ctypes.c_int32)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("gain_ctas_per_sm", ctypes.c_int32),
                ("apply_ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p)]


class RoundStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in STAT_FIELDS]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(PHASES)), ("launches", ctypes.c_int64 * len(PHASES))]


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Loads libhgp.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libhgp.so not built ({_LIB_PATH}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(_LIB_PATH)
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.hgp_default_options.argtypes = [P]
        lib.hgp_default_options.restype = None
        lib.hgp_strerror.argtypes = [ctypes.c_int]
        lib.hgp_strerror.restype = ctypes.c_char_p
        for name in ("hgp_create", "hgp_create_device"):
            fn = getattr(lib, name)
            fn.argtypes = [i32, i32, P, P, P, P, i32, f64, P, P, P]
            fn.restype = ctypes.c_int
        lib.hgp_refine.argtypes = [P, i32, P]
        lib.hgp_set_partition.argtypes = [P, P, i32]
        lib.hgp_objective.argtypes = [P, P]
        lib.hgp_objective_from_phi.argtypes = [P, P]
        lib.hgp_get_partition.argtypes = [P, P, i32]
        lib.hgp_get_block_weights.argtypes = [P, P]
        lib.hgp_get_phi.argtypes = [P, P]
        lib.hgp_get_lambda.argtypes = [P, P]
        lib.hgp_get_info.argtypes = [P, P, P, P, P, P, P, P, P]
        lib.hgp_debug_candidates.argtypes = [P, i32, P, P]
        lib.hgp_exact_gains.argtypes = [P, i32, P, P]
        lib.hgp_rebalance.argtypes = [P, i32, P, P, P]
        lib.hgp_set_launch_shape.argtypes = [P, i32, i32]
        lib.hgp_contract.argtypes = [i32, i32, P, P, P, P, P, P, P]
        lib.hgp_coarse_get_sizes.argtypes = [P, P, P, P]
        lib.hgp_coarse_get_device_arrays.argtypes = [P, P, P, P, P, P]
        lib.hgp_coarse_copy_to_host.argtypes = [P, P, P, P, P, P]
        lib.hgp_coarse_project.argtypes = [P, P, P]
        lib.hgp_coarse_destroy.argtypes = [P]
        lib.hgp_coarse_destroy.restype = None
        lib.hgp_exact_gains.restype = ctypes.c_int
        lib.hgp_export_state.argtypes = [P, P, P, P, P]
        lib.hgp_import_state.argtypes = [P, P, P, i64, i32]
        lib.hgp_export_state.restype = ctypes.c_int
        lib.hgp_import_state.restype = ctypes.c_int
        lib.hgp_set_profiling.argtypes = [P, i32]
        lib.hgp_get_profile.argtypes = [P, P]
        lib.hgp_get_launch_count.argtypes = [P, P]
        for name in ("hgp_refine", "hgp_set_partition", "hgp_objective", "hgp_objective_from_phi",
                     "hgp_get_partition", "hgp_get_block_weights", "hgp_get_phi", "hgp_get_lambda",
                     "hgp_get_info", "hgp_debug_candidates", "hgp_set_profiling",
                     "hgp_get_profile", "hgp_get_launch_count"):
            getattr(lib, name).restype = ctypes.c_int
        lib.hgp_candidates_noalloc.argtypes = [i32, i32, P, P, P, P, P, P, i32, f64, P, i32,
                                               ctypes.c_uint64, i32, P, P, P]
        lib.hgp_candidates_noalloc.restype = ctypes.c_int
        lib.hgp_batch_default_options.argtypes = [P]
        lib.hgp_batch_default_options.restype = None
        lib.hgp_batch_create.argtypes = [P, i32, P, P]
        lib.hgp_batch_refine.argtypes = [P, i32, P]
        lib.hgp_batch_synchronize.argtypes = [P]
        lib.hgp_batch_get_launch_count.argtypes = [P, P]
        lib.hgp_batch_get_stats.argtypes = [P, i32, P]
        lib.hgp_batch_query.argtypes = [P, P]
        lib.hgp_batch_get_partitions.argtypes = [P, P, i32, P]
        lib.hgp_set_blocking_waits.argtypes = [i32]
        lib.hgp_set_blocking_waits.restype = ctypes.c_int
        for name in ("hgp_batch_create", "hgp_batch_refine", "hgp_batch_synchronize",
                     "hgp_batch_get_launch_count", "hgp_batch_get_stats", "hgp_batch_query",
                     "hgp_batch_get_partitions"):
            getattr(lib, name).restype = ctypes.c_int
        lib.hgp_set_pool_retention.argtypes = [i64]
        lib.hgp_set_pool_retention.restype = ctypes.c_int
        lib.hgp_batch_destroy.argtypes = [P]
        lib.hgp_batch_destroy.restype = None
        lib.hgp_probe_gather.argtypes = [i64, i64, P, P]
        lib.hgp_probe_gather.restype = ctypes.c_int
        lib.hgp_probe_atomic.argtypes = [i64, i64, P, P]
        lib.hgp_probe_atomic.restype = ctypes.c_int
        lib.hgp_destroy.argtypes = [P]
        lib.hgp_destroy.restype = None
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load_library().hgp_strerror(int(code)).decode()
    except ImportError:
        return "library not loaded"


def default_options() -> Options:
    o = Options()
    load_library().hgp_default_options(ctypes.byref(o))
    return o


def _check(code: int, what: str):
    if code != HGP_OK:
        raise HGPError(code, what)


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _hptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _dptr(t):
    if t is None:
        return None
    if isinstance(t, int):          # a raw device pointer (e.g. one owned by a Coarse)
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(int(t.data_ptr()))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class HGP:
    """One hypergraph + partition resident on the GPU (a handle of libhgp).

    Host inputs are numpy arrays: net_off int64[m+1], pins int32[P], part int32[n],
    vertex_w / net_w int32 or None.  With ``device=True`` every array is a torch CUDA tensor
    of the same dtype instead.
    """

    def __init__(self, n, m, net_off, pins, k, eps, part, vertex_w=None, net_w=None, *,
                 subrounds: int = 4, seed: int = 0, phi_width: int = 0, debug: int = 0,
                 graph: int = 0, stream=None, device: bool = False, balance_moves: bool = False,
                 revert_negative: bool = False, gain_ctas_per_sm: int = 0, apply_ctas_per_sm: int = 0):
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        o = default_options()
        o.subrounds, o.phi_width, o.seed = int(subrounds), int(phi_width), int(seed)
        o.debug, o.graph = int(debug), int(graph)
        o.balance_moves, o.revert_negative = int(bool(balance_moves)), int(bool(revert_negative))
        o.gain_ctas_per_sm, o.apply_ctas_per_sm = int(gain_ctas_per_sm), int(apply_ctas_per_sm)
        sh = _stream_handle(stream)
        o.cuda_stream = ctypes.c_void_p(sh) if sh else None
        self.n, self.m, self.k = int(n), int(m), int(k)
        if device:
            args = [_dptr(net_off), _dptr(pins), _dptr(vertex_w), _dptr(net_w)]
            pt = _dptr(part)
            fn = self._lib.hgp_create_device
        else:
            keep = [_host(net_off, np.int64), _host(pins, np.int32), _host(vertex_w, np.int32),
                    _host(net_w, np.int32), _host(part, np.int32)]
            args = [_hptr(x) for x in keep[:4]]
            pt = _hptr(keep[4])
            fn = self._lib.hgp_create
        rc = fn(self.n, self.m, *args, self.k, float(eps), pt, ctypes.byref(o), ctypes.byref(self._h))
        _check(rc, "hgp_create")

    @classmethod
    def from_hypergraph(cls, hg, part=None, **kw):
        return cls(hg.n, hg.m, hg.net_off, hg.pins, hg.k, hg.eps,
                   hg.part if part is None else part, hg.vertex_w, hg.net_w, **kw)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.hgp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- refinement
    def refine(self, rounds: int, stats: bool = True):
        """Runs `rounds` LP rounds; returns int64 [rounds x 7] statistics (STAT_FIELDS) or None."""
        if stats:
            buf = (RoundStats * max(1, rounds))()
            _check(self._lib.hgp_refine(self._h, int(rounds), buf), "hgp_refine")
            return np.array([[getattr(buf[i], f) for f in STAT_FIELDS] for i in range(rounds)],
                            dtype=np.int64).reshape(rounds, len(STAT_FIELDS))
        _check(self._lib.hgp_refine(self._h, int(rounds), None), "hgp_refine")
        return None

    def set_partition(self, part, device: bool = False):
        if device:
            _check(self._lib.hgp_set_partition(self._h, _dptr(part), 1), "hgp_set_partition")
        else:
            p = _host(part, np.int32)
            _check(self._lib.hgp_set_partition(self._h, _hptr(p), 0), "hgp_set_partition")

    # -- results
    def objective(self) -> int:
        out = ctypes.c_int64()
        _check(self._lib.hgp_objective(self._h, ctypes.byref(out)), "hgp_objective")
        return out.value

    def objective_from_phi(self) -> int:
        out = ctypes.c_int64()
        _check(self._lib.hgp_objective_from_phi(self._h, ctypes.byref(out)), "hgp_objective_from_phi")
        return out.value

    def partition(self, out_device=None, out=None) -> Optional[np.ndarray]:
        """The partition as int32[n]: into the device tensor out_device, into the host array
        `out` (e.g. page-locked, for a faster copy), or into a new numpy array."""
        if out_device is not None:
            _check(self._lib.hgp_get_partition(self._h, _dptr(out_device), 1), "hgp_get_partition")
            return None
        if out is None:
            out = np.empty(self.n, dtype=np.int32)
        elif out.dtype != np.int32 or out.size < self.n or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous int32 array of at least n entries")
        _check(self._lib.hgp_get_partition(self._h, _hptr(out), 0), "hgp_get_partition")
        return out

    def block_weights(self) -> np.ndarray:
        out = np.empty(self.k, dtype=np.int64)
        _check(self._lib.hgp_get_block_weights(self._h, _hptr(out)), "hgp_get_block_weights")
        return out

    def phi(self) -> np.ndarray:
        out = np.empty((self.m, self.k), dtype=np.int32)
        _check(self._lib.hgp_get_phi(self._h, _hptr(out)), "hgp_get_phi")
        return out

    def lam(self) -> np.ndarray:
        out = np.empty(self.m, dtype=np.uint64)
        _check(self._lib.hgp_get_lambda(self._h, _hptr(out)), "hgp_get_lambda")
        return out

    def info(self) -> dict:
        vals = [ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(),
                ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()]
        _check(self._lib.hgp_get_info(self._h, *[ctypes.byref(v) for v in vals]), "hgp_get_info")
        keys = ("n", "m", "k", "pins", "lmax", "phi_width", "wide_nets", "next_round")
        return {kk: v.value for kk, v in zip(keys, vals)}

    def debug_candidates(self, s: int):
        t = np.empty(self.n, dtype=np.int32)
        g = np.empty(self.n, dtype=np.int64)
        _check(self._lib.hgp_debug_candidates(self._h, int(s), _hptr(t), _hptr(g)),
               "hgp_debug_candidates")
        return t, g

    def set_launch_shape(self, gain_ctas_per_sm: int = 0, apply_ctas_per_sm: int = 0):
        _check(self._lib.hgp_set_launch_shape(self._h, int(gain_ctas_per_sm), int(apply_ctas_per_sm)),
               "hgp_set_launch_shape")

    def rebalance(self, max_passes: int):
        """Rebalancing passes (Sec. 8); returns (stats [passes x 7] int64 (STAT_FIELDS),
        phases [passes] int32)."""
        buf = (RoundStats * max(1, max_passes))()
        ph = np.zeros(max(1, max_passes), dtype=np.int32)
        n = ctypes.c_int32(0)
        _check(self._lib.hgp_rebalance(self._h, int(max_passes), buf, _hptr(ph), ctypes.byref(n)),
               "hgp_rebalance")
        p = n.value
        st = np.array([[getattr(buf[i], f) for f in STAT_FIELDS] for i in range(p)],
                      dtype=np.int64).reshape(p, len(STAT_FIELDS))
        return st, ph[:p].copy()

    def exact_gains(self, moves) -> np.ndarray:
        """Gains of a move sequence [(u, from, to), ...] performed in order (Lemma 1)."""
        mv = np.ascontiguousarray(moves, dtype=np.int32).reshape(-1, 3)
        g = np.empty(mv.shape[0], dtype=np.int64)
        _check(self._lib.hgp_exact_gains(self._h, int(mv.shape[0]), _hptr(mv), _hptr(g)), "hgp_exact_gains")
        return g

    # -- checkpoint / resume
    def export_state(self) -> dict:
        part = np.empty(self.n, dtype=np.int32)
        moved = np.empty(max(1, self.m), dtype=np.uint8)
        r, first = ctypes.c_int64(), ctypes.c_int32()
        _check(self._lib.hgp_export_state(self._h, _hptr(part), _hptr(moved), ctypes.byref(r),
                                          ctypes.byref(first)), "hgp_export_state")
        return {"partition": part, "moved_nets": moved[:self.m], "next_round": r.value,
                "first_round": first.value}

    def import_state(self, state: dict):
        part = _host(state["partition"], np.int32)
        moved = _host(state.get("moved_nets"), np.uint8)
        _check(self._lib.hgp_import_state(self._h, _hptr(part), _hptr(moved),
                                          int(state["next_round"]), int(state["first_round"])),
               "hgp_import_state")

    # -- measurement
    def set_profiling(self, enable: bool = True):
        _check(self._lib.hgp_set_profiling(self._h, 1 if enable else 0), "hgp_set_profiling")

    def profile(self) -> dict:
        p = Profile()
        _check(self._lib.hgp_get_profile(self._h, ctypes.byref(p)), "hgp_get_profile")
        return {name: (p.ms[i], p.launches[i]) for i, name in enumerate(PHASES)}

    def launch_count(self) -> int:
        out = ctypes.c_int64()
        _check(self._lib.hgp_get_launch_count(self._h, ctypes.byref(out)), "hgp_get_launch_count")
        return out.value


def candidates_noalloc(n, m, net_off, pins, vtx_off, inc, k, eps, part, target, gain,
                       vertex_w=None, net_w=None, subrounds: int = 4, seed: int = 0, s: int = 0,
                       stream=None):
    """hgp_candidates_noalloc on torch CUDA tensors (int32 inputs, int32 target, int64 gain).
    Returns the status code (0 = success)."""
    lib = load_library()
    sh = _stream_handle(stream)
    return int(lib.hgp_candidates_noalloc(
        int(n), int(m), _dptr(net_off), _dptr(pins), _dptr(vtx_off), _dptr(inc), _dptr(vertex_w),
        _dptr(net_w), int(k), float(eps), _dptr(part), int(subrounds), int(seed), int(s),
        _dptr(target), _dptr(gain), ctypes.c_void_p(sh) if sh else None))


class Batch:
    """hgp_batch over existing HGP handles (which must stay alive while the batch is used)."""

    def __init__(self, handles, graph: bool = True, gain_ctas_per_sm: int = 0,
                 apply_ctas_per_sm: int = 0, stream=None):
        self._lib = load_library()
        self.handles = list(handles)
        o = BatchOptions()
        self._lib.hgp_batch_default_options(ctypes.byref(o))
        o.graph = 1 if graph else 0
        o.gain_ctas_per_sm, o.apply_ctas_per_sm = int(gain_ctas_per_sm), int(apply_ctas_per_sm)
        sh = _stream_handle(stream)
        o.cuda_stream = ctypes.c_void_p(sh) if sh else None
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        self._b = ctypes.c_void_p()
        _check(self._lib.hgp_batch_create(arr, len(self.handles), ctypes.byref(o),
                                          ctypes.byref(self._b)), "hgp_batch_create")

    def refine(self, rounds: int, stats: bool = True):
        """Runs `rounds` rounds on every member; returns int64 [count x rounds x 7] or None
        (then the call returns with the work queued; see stats())."""
        n = len(self.handles)
        if stats:
            buf = (RoundStats * max(1, n * rounds))()
            _check(self._lib.hgp_batch_refine(self._b, int(rounds), buf), "hgp_batch_refine")
            return _stats_array(buf, n * rounds).reshape(n, rounds, len(STAT_FIELDS))
        _check(self._lib.hgp_batch_refine(self._b, int(rounds), None), "hgp_batch_refine")
        return None

    def partitions(self, members):
        """Partitions of the listed members (indices into handles) after the last refine call,
        with one copy and one wait: a list of int32 arrays."""
        idx = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
        sizes = [self.handles[i].n for i in idx.tolist()]
        out = np.empty(int(sum(sizes)), dtype=np.int32)
        _check(self._lib.hgp_batch_get_partitions(self._b, idx.ctypes.data_as(ctypes.c_void_p), int(idx.size),
                                                  out.ctypes.data_as(ctypes.c_void_p)), "hgp_batch_get_partitions")
        return np.split(out, np.cumsum(sizes)[:-1]) if sizes else []

    def done(self) -> bool:
        """Whether the last refine call has finished on the device (does not block)."""
        d = ctypes.c_int32(0)
        _check(self._lib.hgp_batch_query(self._b, ctypes.byref(d)), "hgp_batch_query")
        return bool(d.value)

    def stats(self, rounds: int):
        """Statistics of the last refine call (of `rounds` rounds), waiting for that call
        only: int64 [count x rounds x 7]."""
        n = len(self.handles)
        buf = (RoundStats * max(1, n * rounds))()
        _check(self._lib.hgp_batch_get_stats(self._b, int(rounds), buf), "hgp_batch_get_stats")
        return _stats_array(buf, n * rounds).reshape(n, rounds, len(STAT_FIELDS))

    def synchronize(self):
        _check(self._lib.hgp_batch_synchronize(self._b), "hgp_batch_synchronize")

    def launch_count(self) -> int:
        out = ctypes.c_int64()
        _check(self._lib.hgp_batch_get_launch_count(self._b, ctypes.byref(out)), "hgp_batch_get_launch_count")
        return out.value

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self._lib.hgp_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stats_array(buf, count: int) -> np.ndarray:
    raw = np.frombuffer(buf, dtype=np.int64, count=count * len(STAT_FIELDS))
    return raw.reshape(count, len(STAT_FIELDS)).copy()


def set_pool_retention(nbytes: int):
    """hgp_set_pool_retention: freed device memory the library's pool of the current device
    keeps for reuse (0 = give it back at the next synchronisation)."""
    _check(load_library().hgp_set_pool_retention(int(nbytes)), "hgp_set_pool_retention")


def set_blocking_waits(on: bool):
    """hgp_set_blocking_waits: the library's host waits sleep on blocking-sync events (True)
    or spin (False, the default).  Process-wide."""
    _check(load_library().hgp_set_blocking_waits(1 if on else 0), "hgp_set_blocking_waits")


def probe_gather(array_bytes: int = 1600 << 20, n_gathers: int = 86_000_000):
    """Random 32-byte gather rate of the current device: (ms, gathers per second)."""
    lib = load_library()
    ms, rate = ctypes.c_double(), ctypes.c_double()
    _check(lib.hgp_probe_gather(int(array_bytes), int(n_gathers), ctypes.byref(ms), ctypes.byref(rate)),
           "hgp_probe_gather")
    return ms.value, rate.value


def probe_atomic(array_bytes: int = 6400 << 20, n_atomics: int = 50_000_000):
    """Random 32-bit atomic-add rate (old value consumed) of the current device: (ms, atomics
    per second)."""
    lib = load_library()
    ms, rate = ctypes.c_double(), ctypes.c_double()
    _check(lib.hgp_probe_atomic(int(array_bytes), int(n_atomics), ctypes.byref(ms), ctypes.byref(rate)),
           "hgp_probe_atomic")
    return ms.value, rate.value


class Coarse:
    """hgp_contract over device arrays (torch CUDA tensors): the coarse hypergraph of a
    clustering (Sec. 3.2), owned on the device until close()."""

    def __init__(self, n, m, net_off, pins, vertex_w, net_w, cluster, stream=None):
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        self.fine_n = int(n)
        sh = _stream_handle(stream)
        _check(self._lib.hgp_contract(int(n), int(m), _dptr(net_off), _dptr(pins), _dptr(vertex_w),
                                      _dptr(net_w), _dptr(cluster), ctypes.c_void_p(sh) if sh else None,
                                      ctypes.byref(self._h)), "hgp_contract")
        n2, m2, p2 = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(self._lib.hgp_coarse_get_sizes(self._h, ctypes.byref(n2), ctypes.byref(m2), ctypes.byref(p2)),
               "hgp_coarse_get_sizes")
        self.n, self.m, self.num_pins = n2.value, m2.value, p2.value

    def device_arrays(self) -> dict:
        """Raw device pointers (ints) owned by this object."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        _check(self._lib.hgp_coarse_get_device_arrays(self._h, *[ctypes.byref(p) for p in ptrs]),
               "hgp_coarse_get_device_arrays")
        return dict(zip(("net_off", "pins", "vertex_w", "net_w", "map"), (p.value or 0 for p in ptrs)))

    def to_host(self) -> dict:
        out = {"n": self.n, "m": self.m, "net_off": np.empty(self.m + 1, np.int64),
               "pins": np.empty(max(1, self.num_pins), np.int32), "vertex_w": np.empty(max(1, self.n), np.int32),
               "net_w": np.empty(max(1, self.m), np.int32), "map": np.empty(self.fine_n, np.int32)}
        _check(self._lib.hgp_coarse_copy_to_host(self._h, _hptr(out["net_off"]), _hptr(out["pins"]),
                                                 _hptr(out["vertex_w"]), _hptr(out["net_w"]), _hptr(out["map"])),
               "hgp_coarse_copy_to_host")
        out["pins"] = out["pins"][:self.num_pins]
        out["vertex_w"] = out["vertex_w"][:self.n]
        out["net_w"] = out["net_w"][:self.m]
        return out

    def handle(self, k, eps, part, **kw) -> "HGP":
        """An HGP over the coarse arrays (no copy through the host); part: device int32[n']."""
        a = self.device_arrays()
        return HGP(self.n, self.m, a["net_off"], a["pins"], k, eps, part, a["vertex_w"], a["net_w"],
                   device=True, **kw)

    def project(self, coarse_part, fine_part):
        """fine_part[u] = coarse_part[map[u]] (device int32 tensors)."""
        _check(self._lib.hgp_coarse_project(self._h, _dptr(coarse_part), _dptr(fine_part)), "hgp_coarse_project")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.hgp_coarse_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
