#!/usr/bin/env python
"""Benchmark of GPU label-propagation refinement (LP-refine pins/s per round).

A step is one refinement of `rounds` synchronous LP rounds (every row of the hot path:
sub-round lists, gain + best target, approval, apply with Phi/Lambda/objective update) of
the whole instance, started from the instance's start partition.  The partition is reset on
the device between steps, outside the timed region.  value = pins x rounds / step time,
i.e. P divided by the mean wall time of one round, summed over ranks (replicas).

Default workload: the large power-law instance (n = m = 5*10^7, |e| = min(2 + Zipf(2.1),
10^5), k = 64, net weights U{1..10}, 5 rounds), ~3.4*10^8 pins, far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload powerlaw|rownet|small]
  python bench.py --impl reference     # the CPU oracle on a bounded sample, same metric
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "LP-refine pins/s per round, % HBM roofline; batched vs plain; p50/p99 latency"
UNIT = "pins/s"
CACHE = os.environ.get("HGP_SYNTH_CACHE", "/tmp/hgp_synth_cache")
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "powerlaw": (synth.config_powerlaw, "power-law n=m=5e7 |e|=min(2+Zipf(2.1),1e5) k=64 omega=U{1..10}"),
    "rownet": (synth.config_rownet, "row-net 2e6 x 2e6 nnz/row=1+Poisson(9) banded k=8"),
    "small": (synth.config_small, "planted n=m=1e4 k=2 |e|=2+Poisson(4)"),
}
# bounded oracle sample per workload: same recipe, smaller scale
SAMPLE_SCALE = {"powerlaw": 0.01, "rownet": 0.1, "small": 1.0}


# ------------------------------------------------------------------------------ inputs
def load_instance(name: str, scale: float):
    os.makedirs(CACHE, exist_ok=True)
    path = os.path.join(CACHE, f"{name}_{scale:g}.npz")
    fn = WORKLOADS[name][0]
    if os.path.exists(path):
        try:
            z = np.load(path, allow_pickle=False)
            meta = json.loads(str(z["meta"]))
            return synth.Hypergraph(meta["name"], meta["n"], meta["m"], meta["k"], meta["eps"],
                                    z["net_off"], z["pins"], z["part"],
                                    z["vertex_w"] if "vertex_w" in z.files else None,
                                    z["net_w"] if "net_w" in z.files else None, meta["rounds"])
        except Exception:
            pass
    hg = fn(scale=scale)
    arrays = {"net_off": hg.net_off, "pins": hg.pins, "part": hg.part}
    if hg.vertex_w is not None:
        arrays["vertex_w"] = hg.vertex_w
    if hg.net_w is not None:
        arrays["net_w"] = hg.net_w
    meta = dict(n=hg.n, m=hg.m, k=hg.k, eps=hg.eps, rounds=hg.rounds, name=hg.name)
    try:
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, meta=json.dumps(meta), **arrays)
        os.replace(tmp, path)
    except OSError:
        pass
    return hg


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------ helpers
def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(hg, info, stats, S):
    """Algorithmic bytes per launch of the gain and apply kernels (the data the method must
    move, without sector over-fetch), averaged over the launches of one refinement.

    gain, per active vertex: vtx_off 4 B + Pi 1 B + c 4 B (0 if unit); per visited
    incidence: net id 4 B + omega 4 B (0 if unit) + Lambda ceil(k/8) B rounded to 4 or 8
    + Phi(e,a) w B + moved flag 1 B.  Every vertex is active once per round and visits all
    its incidences, so one round = n vertices and P incidences.
    apply, per approved move: Pi write 1 B + 2 block-weight atomics 16 B + candidate 8 B;
    per moved incidence: net id 4 B + Phi(e,a), Phi(e,t) read+write 4w B + Lambda/S1
    read-modify-write 2 x 2 x lam B + moved flag 1 B.
    """
    k, w = info["k"], info["phi_width"]
    lam = 4 if k <= 32 else 8
    per_vertex = 4 + 1 + (4 if hg.vertex_w is not None else 0)
    per_inc = 4 + (4 if hg.net_w is not None else 0) + lam + w + 1
    rounds = stats.shape[0]
    gain_total = rounds * (hg.n * per_vertex + info["pins"] * per_inc)
    moved_pins = int(stats[:, 5].sum())
    approved = int(stats[:, 2].sum())
    apply_total = approved * (1 + 16 + 8) + moved_pins * (4 + 4 * w + 4 * lam + 1)
    launches = rounds * S
    return {"gain": gain_total / launches, "apply": apply_total / launches}


def source_sha256() -> str:
    """sha256 of the sources the profiled kernels and their data layout come from."""
    csrc = os.path.join(ROOT, "paper_2010_10272_gb300", "csrc")
    d = hashlib.sha256()
    for f in ("hgp_refine.cu", "hgp_setup.cu"):
        d.update(open(os.path.join(csrc, f), "rb").read())
    return d.hexdigest()


def traffic_from_profile(kernel: str, workload: str, phi_width: int):
    """dram bytes per launch recorded in profiles/ for `kernel` on `workload`, if the kernel
    sources have not changed since the capture (the sha256 of hgp_refine.cu followed by
    hgp_setup.cu, which decides the data layout, is stored with the figure) and the capture
    used the same Phi entry width."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    pw = re.search(r"phi_width:\s*(\d+)", text)
    if not pw or int(pw.group(1)) != phi_width:
        return None
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256[^:\n]*:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    if source_sha256() != h.group(1):
        return None
    return float(m.group(1))


L2_FLUSH_BYTES = 256 << 20   # twice the GB300's L2


class L2Flush:
    """Writes a buffer twice the size of L2 on the current stream, so that a timed step starts
    with nothing of the instance in L2."""

    def __init__(self, dev):
        import torch
        self.buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def __call__(self):
        self.buf.fill_(1)


def set_l2_fetch_granularity(nbytes: int):
    """Measurement option: the current context's maximum L2 fetch granularity (32..128 bytes;
    CU_LIMIT_MAX_L2_FETCH_GRANULARITY through the driver API).  It lasts as long as the
    context, i.e. this process, and applies to every kernel in it."""
    import ctypes
    import torch
    torch.zeros(1, device="cuda")                 # the context exists from here on
    cuda = ctypes.CDLL("libcuda.so.1")
    rc = cuda.cuCtxSetLimit(ctypes.c_int(5), ctypes.c_size_t(int(nbytes)))
    got = ctypes.c_size_t(0)
    cuda.cuCtxGetLimit(ctypes.byref(got), ctypes.c_int(5))
    if rc != 0 or got.value != nbytes:
        raise RuntimeError(f"could not set the L2 fetch granularity to {nbytes} (rc {rc}, now {got.value})")


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() and args.impl != "reference" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------ oracle
def variant_kwargs(name: str) -> dict:
    return {"balance_moves": "balance" in name, "revert_negative": "revert" in name}


def oracle_sample(workload: str, steps: int, warmup: int, rounds_override=None, variant="plain"):
    """Times the CPU oracle (single thread) on a bounded sample of the workload: the same
    recipe at a smaller scale, `rounds` rounds per step from the start partition."""
    import oracle
    scale = SAMPLE_SCALE[workload]
    hg = load_instance(workload, scale)
    rounds = rounds_override or hg.rounds
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        o = oracle.Oracle.from_hypergraph(hg, subrounds=4, **variant_kwargs(variant))
        t1 = time.perf_counter()
        o.refine(rounds)
        t2 = time.perf_counter()
        o.close()
        if i >= warmup:
            times.append(t2 - t1)
    per_step = statistics.mean(times)
    value = hg.num_pins * rounds / per_step
    sample = (f"{hg.name}: P={hg.num_pins} pins, {rounds} rounds per step from the start "
              f"partition (scale {scale:g} of the workload), oracle creation excluded")
    return value, per_step, sample, hg


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    if args.workload in ("batch", "serving", "rebalance", "contract"):
        args.workload = "small"
    value, per_step, sample, hg = oracle_sample(args.workload, args.steps, args.warmup,
                                                variant=args.variant)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1], "sample": sample, "rounds": hg.rounds,
                   "subrounds": 4, "variant": args.variant},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
def run_gpu(args, world, rank, local):
    import torch
    from paper_2010_10272_gb300 import HGP, build
    from paper_2010_10272_gb300.native import set_pool_retention
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.l2_fetch_granularity:
        set_l2_fetch_granularity(args.l2_fetch_granularity)

    t_gen = time.perf_counter()
    hg = load_instance(args.workload, args.scale)
    t_gen = time.perf_counter() - t_gen
    R, S = hg.rounds, args.subrounds
    P = hg.num_pins

    to_dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d_off, d_pins, d_part = to_dev(hg.net_off), to_dev(hg.pins), to_dev(hg.part)
    d_vw, d_nw = to_dev(hg.vertex_w), to_dev(hg.net_w)
    # one explicit stream for the library and the timing events (a NULL stream handle would
    # make the library create its own stream)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    variant = variant_kwargs(args.variant)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    h = HGP(hg.n, hg.m, d_off, d_pins, hg.k, hg.eps, d_part, d_vw, d_nw, subrounds=S, device=True,
            stream=stream, **variant)
    info = h.info()
    torch.cuda.synchronize()
    state_bytes = free_before - torch.cuda.mem_get_info()[0]   # what the handle holds on the device
    del d_off, d_pins, d_vw, d_nw

    flush = L2Flush(dev)

    def step(timed_events=None):
        h.set_partition(d_part, device=True)
        flush()
        torch.cuda.synchronize()
        barrier(world)
        if timed_events is not None:
            timed_events[0].record(stream)
        st = h.refine(R)
        if timed_events is not None:
            timed_events[1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return st

    for _ in range(args.warmup):
        step()

    sampler = ClockSampler(local)
    sampler.start()
    h.set_profiling(True)
    ms, launches, stats = [], 0, None
    for _ in range(args.steps):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        l0 = h.launch_count()
        st = step(ev)
        launches += h.launch_count() - l0
        ms.append(ev[0].elapsed_time(ev[1]))
        stats = st
    clocks = sampler.stop()
    prof = h.profile()
    h.set_profiling(False)

    total_ms = max_over_ranks(sum(ms), world)
    value = world * args.steps * P * R / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # roofline of the dominant kernel (gain or apply), from the live per-phase events
    algo = algorithmic_bytes(hg, info, stats, S)
    peak, peak_kind = measured_peak_hbm()
    kern = max(("gain", "apply"), key=lambda kk: prof[kk][0])
    kname = {"gain": "k_gain", "apply": "k_apply"}[kern]
    avg_ms = prof[kern][0] / max(1, prof[kern][1])
    achieved = algo[kern] / (avg_ms / 1e3) / 1e9
    traffic = traffic_from_profile(kname, args.workload, info["phi_width"])
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                "traffic": traffic, "algorithmic_bytes_per_launch": algo[kern],
                "avg_launch_ms": avg_ms}
    # DRAM bytes actually moved by the gain and update kernels together (ncu dram__bytes of one
    # launch each, from profiles/) over their live average launch times
    t_gain = traffic_from_profile("k_gain", args.workload, info["phi_width"])
    t_apply = traffic_from_profile("k_apply", args.workload, info["phi_width"])
    if t_gain and t_apply:
        ms_g = prof["gain"][0] / max(1, prof["gain"][1])
        ms_a = prof["apply"][0] / max(1, prof["apply"][1])
        gbs = (t_gain + t_apply) / ((ms_g + ms_a) / 1e3) / 1e9
        roofline["dram_gain_plus_update"] = {"achieved_gbs": gbs, "frac": gbs / peak,
                                             "source": "ncu dram__bytes per launch (profiles/) / live launch time"}
    # second roofline: the gain step is bound by random record gathers (one per incidence of an
    # active vertex), compared with the device's measured random 32-byte gather rate
    from paper_2010_10272_gb300.native import probe_gather
    g_ms, g_rate = probe_gather(1600 << 20, 86_000_000)
    gain_ms = prof["gain"][0] / max(1, prof["gain"][1])
    gathers_per_launch = info["pins"] / S
    roofline["gather"] = {"kernel": "k_gain", "achieved_gathers_per_s": gathers_per_launch / (gain_ms / 1e3),
                          "peak_gathers_per_s": g_rate,
                          "frac": gathers_per_launch / (gain_ms / 1e3) / g_rate,
                          "peak_kind": "measured random 32-byte gathers from a 1.6 GB array (hgp_probe_gather)"}
    # the apply step's ceiling: two pin-count atomics with results per moved incidence, against
    # the device's measured rate of random atomics with results on an array of the Phi table's size
    from paper_2010_10272_gb300.native import probe_atomic
    a_ms_probe, a_rate = probe_atomic(6400 << 20, 50_000_000)
    apply_ms = prof["apply"][0] / max(1, prof["apply"][1])
    atomics_per_launch = 2.0 * float(stats[:, 5].sum()) / (R * S)
    roofline["atomic"] = {"kernel": "k_apply", "achieved_atomics_per_s": atomics_per_launch / (apply_ms / 1e3),
                          "peak_atomics_per_s": a_rate,
                          "frac": atomics_per_launch / (apply_ms / 1e3) / a_rate,
                          "peak_kind": "measured random 32-bit atomics with results on a 6.4 GB array (hgp_probe_atomic)"}
    phases = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
              for k, v in prof.items()}
    other = "apply" if kern == "gain" else "gain"
    o_ms = prof[other][0] / max(1, prof[other][1])
    phases["frac_of_peak_other"] = {"kernel": f"k_{other}",
                                   "achieved_gbs": algo[other] / (o_ms / 1e3) / 1e9,
                                   "frac": algo[other] / (o_ms / 1e3) / 1e9 / peak}

    # end to end through the C ABI with host buffers: create (H2D + setup) + refine + result D2H
    e2e = None
    if not args.no_e2e:
        pin = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hp = [pin(hg.net_off), pin(hg.pins), pin(hg.part), pin(hg.vertex_w), pin(hg.net_w)]
        part_out = pin(np.zeros(hg.n, np.int32))           # page-locked result buffer
        h2d = sum(a.nbytes for a in hp if a is not None)
        d2h = hg.n * 4 + R * 8 * 7
        del h
        torch.cuda.empty_cache()
        # freed device memory stays in the library's pool between steps, as in a process that
        # partitions repeatedly (hgp_set_pool_retention); without it every creation maps its
        # ~15 GB afresh and every destroy unmaps them
        set_pool_retention(args.e2e_pool_retention)
        times = []
        for i in range(1 + args.e2e_steps):
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            h2 = HGP(hg.n, hg.m, hp[0], hp[1], hg.k, hg.eps, hp[2], hp[3], hp[4], subrounds=S,
                     stream=stream, **variant)
            h2.refine(R)
            h2.partition(out=part_out)
            t1 = time.perf_counter()
            h2.close()
            if i > 0:
                times.append(t1 - t0)
        set_pool_retention(0)
        torch.cuda.empty_cache()
        e2e_t = max_over_ranks(statistics.median(times), world)
        e2e = {"value": world * P * R / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_t * 1e3, "steps": args.e2e_steps,
               "statistic": "median over the steps (after one untimed step)",
               "pool_retention_bytes": args.e2e_pool_retention}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cv, cstep, sample, _ = oracle_sample(args.workload, 1, 0, variant=args.variant)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}

    # the metric's other parts, on the same GPU after the power-law instance is released:
    # batched vs plain launches (batch workload) and serving latency (serving workload)
    extra = {}
    if args.workload == "powerlaw" and args.variant == "plain":
        if "h" in locals():
            del h
        torch.cuda.empty_cache()
        if not args.no_batch:
            b = batch_section(args, stream, world)
            extra["batched_vs_plain"] = b
        if not args.no_serving:
            extra["serving"] = serving_section(args, stream)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1], "n": hg.n, "m": hg.m, "pins": P,
                   "k": hg.k, "eps": hg.eps, "rounds": R, "subrounds": S,
                   "phi_width": info["phi_width"], "wide_nets": info["wide_nets"],
                   "lmax": info["lmax"], "variant": args.variant, "parallelism": f"replicas x{world}",
                   "l2": f"L2 flushed before every timed step (a {L2_FLUSH_BYTES >> 20} MiB write); instance state "
                         f"~{state_bytes / 1e9:.2g} GB resident in HBM",
                   "step": f"reset start partition (untimed) + {R} LP rounds"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "phases": phases,
        "rounds_stats": {"objective": stats[:, 0].tolist(), "approved": stats[:, 2].tolist(),
                         "eligible": stats[:, 3].tolist(), "moved_pins": stats[:, 5].tolist(),
                         "reverted": stats[:, 6].tolist()},
        "setup_s": {"generate_or_load": t_gen},
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ batch workload
def batch_section(args, stream, world=1):
    """The 256-instance batch workload (n log-uniform 1e3-2e5, |e| = min(2+Zipf(2.5), 1000),
    k in {2,4,8,16}, c(v) in U{1..4}, 5 rounds): every phase of a round is one launch over all
    instances, replayed as a CUDA graph with an autotuned launch shape, against the same
    instances refined one after another with plain per-instance launches on the same stream.
    Both from device-resident inputs; a step resets every start partition (untimed) and runs
    all rounds of every instance."""
    import torch
    from paper_2010_10272_gb300 import HGP, Batch
    from paper_2010_10272_gb300.autotune import tune_batch
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    insts = synth.config_batch(count=args.batch_count)
    t_gen = time.perf_counter() - t0
    R, S = insts[0].rounds, args.subrounds
    P = sum(h.num_pins for h in insts)
    to_dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    parts = [to_dev(h.part) for h in insts]
    hs = [HGP(h.n, h.m, to_dev(h.net_off), to_dev(h.pins), h.k, h.eps, parts[i], to_dev(h.vertex_w),
              to_dev(h.net_w), subrounds=S, device=True, stream=stream) for i, h in enumerate(insts)]

    flush = L2Flush(torch.device("cuda", torch.cuda.current_device()))

    def reset():
        for h, p in zip(hs, parts):
            h.set_partition(p, device=True)
        flush()
        torch.cuda.synchronize()

    # launch shape of the persistent kernels: tuned on these handles (state restored after)
    reset()
    tuned = tune_batch(hs, rounds=R, stream=stream)
    shape = {"gain_ctas_per_sm": tuned["gain_ctas_per_sm"], "apply_ctas_per_sm": tuned["apply_ctas_per_sm"],
             "candidates_ms": {f"{g}x{a}": round(ms, 3) for (g, a), ms in tuned["ms"].items()}}
    batch = Batch(hs, graph=True, stream=stream, gain_ctas_per_sm=shape["gain_ctas_per_sm"],
                  apply_ctas_per_sm=shape["apply_ctas_per_sm"])

    def plain_step():
        for h in hs:
            h.refine(R, stats=False)

    def batch_step():
        batch.refine(R, stats=False)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            reset()
            fn()
            torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            reset()
            barrier(world)
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            ms.append(ev[0].elapsed_time(ev[1]))
        return ms

    l0 = batch.launch_count()
    ms_b = timed(batch_step, args.batch_steps, 3)
    launches = (batch.launch_count() - l0) // (args.batch_steps + 3) * args.batch_steps
    ms_p = timed(plain_step, max(2, args.batch_steps // 2), 1)
    total_b = max_over_ranks(sum(ms_b), world)
    value = world * len(ms_b) * P * R / (total_b / 1e3)
    plain = world * len(ms_p) * P * R / (max_over_ranks(sum(ms_p), world) / 1e3)
    batch.close()
    for h in hs:
        h.close()
    del parts
    torch.cuda.empty_cache()
    return {
        "workload": f"batch of {len(insts)} planted hypergraphs, n log-uniform 1e3-2e5, "
                    "|e|=min(2+Zipf(2.5),1000), k in {2,4,8,16}, c(v) in U{1..4}",
        "instances": len(insts), "pins": P, "rounds": R, "subrounds": S,
        "batched_pins_per_s": value, "plain_pins_per_s": plain, "ratio": value / plain,
        "batched_ms_per_step": statistics.mean(ms_b), "plain_ms_per_step": statistics.mean(ms_p),
        "steps": len(ms_b), "plain_steps": len(ms_p),
        "step": f"reset all partitions (untimed) + {R} rounds of every instance",
        "l2": f"L2 flushed before every timed step (a {L2_FLUSH_BYTES >> 20} MiB write)",
        "launch_shape": shape, "gpu_launches": launches, "generate_s": t_gen,
    }


def run_batch(args, world, rank, local):
    """The batch workload alone: value = the batched throughput (pins/s per round)."""
    import torch
    from paper_2010_10272_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(torch.device("cuda", local))
    torch.cuda.set_stream(stream)
    args.batch_steps = args.steps
    sampler = ClockSampler(local)
    sampler.start()
    b = batch_section(args, stream, world)
    clocks = sampler.stop()
    line = {
        "metric": METRIC, "value": b["batched_pins_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": b["steps"], "warmup": 3, "ms_per_step": b["batched_ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": b["workload"], "instances": b["instances"], "pins": b["pins"],
                   "rounds": b["rounds"], "subrounds": b["subrounds"], "parallelism": f"replicas x{world}",
                   "step": b["step"], "l2": b["l2"]},
        "batched_vs_plain": {k: b[k] for k in ("batched_pins_per_s", "plain_pins_per_s", "ratio",
                                                "batched_ms_per_step", "plain_ms_per_step")},
        "launch_shape": b["launch_shape"], "gpu_launches": b["gpu_launches"], "clocks": clocks,
        "setup_s": {"generate": b["generate_s"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ rebalancing
def run_rebalance(args, world, rank, local):
    """Rebalancing (Sec. 8) of the power-law instance from an overloaded start: the planted
    partition with a hash-chosen `--skew` fraction of the vertices moved into block 0.  A step
    resets that start (untimed) and runs hgp_rebalance until balanced (at most 64 passes).
    value = pins x passes / s (the unit of an LP round)."""
    import torch
    from paper_2010_10272_gb300 import HGP, build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    t_gen = time.perf_counter()
    hg = load_instance("powerlaw", args.scale)
    t_gen = time.perf_counter() - t_gen
    S, P = args.subrounds, hg.num_pins
    part = hg.part.copy()
    pick = (np.arange(hg.n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)
    part[pick < np.uint64(int(args.skew * (1 << 24)))] = 0
    to_dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d_part = to_dev(part)
    h = HGP(hg.n, hg.m, to_dev(hg.net_off), to_dev(hg.pins), hg.k, hg.eps, d_part, to_dev(hg.vertex_w),
            to_dev(hg.net_w), subrounds=S, device=True, stream=stream)
    info = h.info()
    w0 = h.block_weights()
    max_passes = 64

    def step(ev=None):
        h.set_partition(d_part, device=True)
        torch.cuda.synchronize()
        barrier(world)
        if ev is not None:
            ev[0].record(stream)
        st, ph = h.rebalance(max_passes)
        if ev is not None:
            ev[1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return st, ph

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local)
    sampler.start()
    ms, launches = [], 0
    for _ in range(args.steps):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        l0 = h.launch_count()
        st, ph = step(ev)
        launches += h.launch_count() - l0
        ms.append(ev[0].elapsed_time(ev[1]))
    clocks = sampler.stop()
    passes = int(st.shape[0])
    total_ms = max_over_ranks(sum(ms), world)
    value = world * args.steps * P * passes / (total_ms / 1e3)
    e2e = None
    if not args.no_e2e:
        pin = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hp = [pin(hg.net_off), pin(hg.pins), pin(part), pin(hg.vertex_w), pin(hg.net_w)]
        h2d = sum(a.nbytes for a in hp if a is not None)
        h.close()
        torch.cuda.empty_cache()
        times = []
        for i in range(1 + args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2 = HGP(hg.n, hg.m, hp[0], hp[1], hg.k, hg.eps, hp[2], hp[3], hp[4], subrounds=S, stream=stream)
            st2, _ = h2.rebalance(max_passes)
            out = h2.partition()
            t1 = time.perf_counter()
            h2.close()
            if i > 0:
                times.append(t1 - t0)
            del out
        e2e_t = max_over_ranks(statistics.mean(times), world)
        e2e = {"value": world * P * int(st2.shape[0]) / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": hg.n * 4 + max_passes * (8 * 7 + 4), "ms_per_step": e2e_t * 1e3,
               "steps": args.e2e_steps}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        scale = SAMPLE_SCALE["powerlaw"]
        hs_ = load_instance("powerlaw", scale)
        ps = hs_.part.copy()
        pk = (np.arange(hs_.n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)
        ps[pk < np.uint64(int(args.skew * (1 << 24)))] = 0
        o = oracle.Oracle.from_hypergraph(hs_, subrounds=S, part=ps)
        t0 = time.perf_counter()
        ost, _, _ = o.rebalance(max_passes)
        dt = time.perf_counter() - t0
        o.close()
        cpu = {"value": hs_.num_pins * max(1, ost.shape[0]) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{hs_.name} with the same skew (scale {scale:g}): {ost.shape[0]} passes in {dt:.1f} s"}
    line = {
        "metric": "rebalance pins/s per pass", "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["powerlaw"][1] + f", {args.skew:g} of the vertices moved into block 0",
                   "n": hg.n, "m": hg.m, "pins": P, "k": hg.k, "lmax": info["lmax"], "subrounds": S,
                   "start_heaviest_block": int(w0.max()), "parallelism": f"replicas x{world}",
                   "step": "reset the overloaded start (untimed) + hgp_rebalance until balanced",
                   "l2": "inputs larger than L2"},
        "passes": passes, "phases": ph.tolist(), "moved": st[:, 2].tolist(),
        "heaviest_after_pass": st[:, 4].tolist(), "objective_after_pass": st[:, 0].tolist(),
        "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clocks,
        "setup_s": {"generate_or_load": t_gen},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ contraction
def pair_clustering(n: int, seed: int) -> np.ndarray:
    """Seeded clustering into about n/2 clusters: a permutation cut into consecutive pairs (a
    stand-in for the paper's clustering, which is out of scope)."""
    perm = np.random.default_rng(seed).permutation(n)
    cl = np.empty(n, np.int32)
    cl[perm] = perm[(np.arange(n) // 2) * 2]
    return cl


def run_contract(args, world, rank, local):
    """Contraction (Sec. 3.2) of the power-law instance by a seeded pair clustering, then of the
    result again, down to four levels; a step contracts H0 -> H1 (timed, inputs in HBM).
    value = fine pins contracted per second.  Also: the whole hierarchy refined in one batch
    against the levels refined one after another."""
    import torch
    from paper_2010_10272_gb300 import HGP, Batch, Coarse, build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    t_gen = time.perf_counter()
    hg = load_instance("powerlaw", args.scale)
    t_gen = time.perf_counter() - t_gen
    P = hg.num_pins
    to_dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d = [to_dev(x) for x in (hg.net_off, hg.pins, hg.vertex_w, hg.net_w)]
    cl = to_dev(pair_clustering(hg.n, 1))
    for _ in range(args.warmup):
        Coarse(hg.n, hg.m, *d, cl, stream=stream).close()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ms = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        c = Coarse(hg.n, hg.m, *d, cl, stream=stream)      # synchronises its stream
        ms.append((time.perf_counter() - t0) * 1e3)
        c.close()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(ms), world)
    value = world * args.steps * P / (total_ms / 1e3)
    # bytes a contraction has to move at least: read offsets, pins, cluster ids of the pins and
    # weights; write the remapped pins once, read them for the fingerprints, write the coarse pins
    c1 = Coarse(hg.n, hg.m, *d, cl, stream=stream)
    algo = 8 * (hg.m + 1) + 4 * P * 5 + 4 * hg.n * 3 + 4 * c1.num_pins * 2
    peak, peak_kind = measured_peak_hbm()
    achieved = algo / (total_ms / args.steps / 1e3) / 1e9
    # hierarchy: H0..H3 by repeated pair contraction, refined together in one batch
    levels = [(hg.n, hg.m, d[0], d[1], d[2], d[3])]
    coarse = [c1]
    for lv in range(1, 4):
        a = coarse[-1].device_arrays()
        cur = coarse[-1]
        levels.append((cur.n, cur.m, a["net_off"], a["pins"], a["vertex_w"], a["net_w"]))
        if lv < 3:
            coarse.append(Coarse(cur.n, cur.m, a["net_off"], a["pins"], a["vertex_w"], a["net_w"],
                                 to_dev(pair_clustering(cur.n, 1 + lv)), stream=stream))
    parts = [to_dev((np.arange(L[0]) % hg.k).astype(np.int32)) for L in levels]
    hs = [HGP(L[0], L[1], L[2], L[3], hg.k, hg.eps, parts[i], L[4], L[5], subrounds=4, device=True,
              stream=stream) for i, L in enumerate(levels)]
    R = hg.rounds

    def reset():
        for h, p in zip(hs, parts):
            h.set_partition(p, device=True)
        torch.cuda.synchronize()
    batch = Batch(hs, graph=True, stream=stream)
    hier = {}
    for name, fn in (("batched", lambda: batch.refine(R, stats=False)),
                     ("one_after_another", lambda: [h.refine(R, stats=False) for h in hs])):
        reset()
        fn()
        torch.cuda.synchronize()
        reset()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        hier[name + "_ms"] = ev[0].elapsed_time(ev[1])
    hier["levels"] = [{"n": L[0], "m": L[1]} for L in levels]
    hier["rounds"] = R
    batch.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        scale = SAMPLE_SCALE["powerlaw"]
        hs_ = load_instance("powerlaw", scale)
        t0 = time.perf_counter()
        oracle.contract(hs_.n, hs_.m, hs_.net_off, hs_.pins, hs_.vertex_w, hs_.net_w, pair_clustering(hs_.n, 1))
        dt = time.perf_counter() - t0
        cpu = {"value": hs_.num_pins / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{hs_.name}, pair clustering (scale {scale:g}): {dt:.2f} s"}
    line = {
        "metric": "contraction pins/s", "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS["powerlaw"][1] + ", seeded pair clustering",
                   "n": hg.n, "m": hg.m, "pins": P, "coarse": {"n": c1.n, "m": c1.m, "pins": c1.num_pins},
                   "parallelism": f"replicas x{world}", "step": "hgp_contract H0 -> H1 (inputs in HBM, "
                   "wall clock around the call, which synchronises)", "l2": "inputs larger than L2"},
        "roofline": {"bound": "hbm", "kernel": "hgp_contract (whole call)", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                     "traffic": None, "algorithmic_bytes_per_launch": algo},
        "hierarchy_batch": hier, "cpu_baseline": cpu, "clocks": clocks,
        "setup_s": {"generate_or_load": t_gen},
    }
    for c in coarse:
        c.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ serving workload
def serving_section(args, stream):
    """The serving workload: requests are planted hypergraphs with pins log-uniform in
    1e4-5e6, |e| = 2+Poisson(4), k in {2,4,8,16,32}, 3 rounds each, every one freshly drawn
    (seeded, on the GPU; synth.device), served with continuous batching (serve.Server).  A
    saturated run (every request queued at t = 0) measures the service capacity mu; Poisson
    arrivals at 0.5 mu and 0.8 mu then give latency percentiles (arrival -> partition on the
    host) over `serve_requests` requests after `serve_warmup` warm-up requests of the same
    stream."""
    import torch
    from paper_2010_10272_gb300.serve import Request, Server, latency_summary
    from synth import device as sdev
    gen_s = 0.0

    def make(seed, count, base):
        nonlocal gen_s
        t = time.perf_counter()
        hgs = sdev.serving_requests(seed, count)
        torch.cuda.empty_cache()
        gen_s += time.perf_counter() - t
        return [Request.from_hypergraph(base + i, h) for i, h in enumerate(hgs)]

    def run(reqs, arrivals):
        srv = Server(stream=stream, creators=args.serve_creators, ctas_per_sm=args.serve_ctas,
                     join_at=args.serve_join_at, depth=args.serve_depth,
                     blocking_waits=bool(args.serve_blocking), tick_streams=args.serve_streams)
        order = sorted(range(len(reqs)), key=lambda i: arrivals[i])
        t_start = time.perf_counter()
        nxt, done = 0, []
        while nxt < len(order) or not srv.idle():
            now = time.perf_counter() - t_start
            while nxt < len(order) and arrivals[order[nxt]] <= now:
                srv.submit(reqs[order[nxt]], arrival=t_start + arrivals[order[nxt]])
                nxt += 1
            if srv.idle():
                time.sleep(max(0.0, min(0.001, arrivals[order[nxt]] - now)))
                continue
            done.extend(srv.step())
        t_total = time.perf_counter() - t_start
        ticks = srv.ticks
        srv.close()
        return done, t_total, ticks

    warm = make(args.serve_seed * 1000 + 1, args.serve_warmup, 0)
    run(warm, [0.0] * len(warm))
    del warm
    sat_reqs = make(args.serve_seed * 1000 + 2, args.serve_saturated, 100_000)
    done, t_sat, ticks = run(sat_reqs, [0.0] * len(sat_reqs))
    work = sum(r.num_pins * r.rounds for r in done)
    mu = len(done) / t_sat
    sat = {"requests": len(done), "seconds": t_sat, "ticks": ticks, "latency": latency_summary(done),
           "pin_rounds_per_s": work / t_sat, "pins": sum(r.num_pins for r in done)}
    del sat_reqs, done
    rng = np.random.default_rng(args.serve_seed)
    rates = {}
    for j, frac in enumerate((0.5, 0.8)):
        lam = frac * mu
        count = args.serve_warmup + args.serve_requests
        reqs = make(args.serve_seed * 1000 + 3 + j, count, 1_000_000 * (j + 1))
        arr = np.cumsum(rng.exponential(1.0 / lam, size=count)).tolist()
        d2, t2, ticks2 = run(reqs, arr)
        measured = [r for r in d2 if r.rid - 1_000_000 * (j + 1) >= args.serve_warmup]
        rates[f"{frac:g}mu"] = dict(latency_summary(measured), arrival_rate_per_s=lam,
                                    warmup_requests=args.serve_warmup, ticks=ticks2,
                                    pin_rounds_per_s=sum(r.num_pins * r.rounds for r in d2) / t2)
        del reqs, d2, measured
    return {
        "workload": "Poisson arrivals of planted hypergraphs, pins log-uniform 1e4-5e6, "
                    "|e|=2+Poisson(4), k in {2,4,8,16,32}, 3 rounds each, every request distinct",
        "service_capacity_req_per_s": mu, "saturated_pin_rounds_per_s": sat["pin_rounds_per_s"],
        "saturated": sat, "poisson": rates, "generate_s": gen_s,
        "server": {"creators": args.serve_creators, "ctas_per_sm": args.serve_ctas, "join_at": args.serve_join_at,
                   "depth": args.serve_depth, "blocking_waits": bool(args.serve_blocking),
                   "tick_streams": args.serve_streams},
        "latency": "arrival -> partition on the host",
    }


def run_serving(args, world, rank, local):
    """The serving workload alone: value = saturated pin-rounds/s."""
    import torch
    from paper_2010_10272_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(torch.device("cuda", local))
    torch.cuda.set_stream(stream)
    sampler = ClockSampler(local)
    sampler.start()
    sv = serving_section(args, stream)
    clocks = sampler.stop()
    sat = sv["saturated"]
    line = {
        "metric": METRIC, "value": sv["saturated_pin_rounds_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": sat["requests"], "warmup": args.serve_warmup, "ms_per_step": sat["seconds"] * 1e3 / sat["requests"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "serving: " + sv["workload"], "requests": sat["requests"],
                   "step": "one request, arrival to partition on the host",
                   "l2": "request state resident in HBM; saturated run", "parallelism": "replicas x1"},
        "serving": sv, "clocks": clocks, "setup_s": {"generate": sv["generate_s"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch", "serving", "rebalance", "contract"],
                    default="powerlaw")
    ap.add_argument("--skew", type=float, default=0.2,
                    help="rebalance workload: fraction of the vertices moved into block 0")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="serving: measured requests per arrival rate (after --serve-warmup)")
    ap.add_argument("--serve-warmup", type=int, default=100)
    ap.add_argument("--serve-saturated", type=int, default=1000,
                    help="serving: requests of the saturated run that measures the capacity")
    ap.add_argument("--serve-seed", type=int, default=1)
    ap.add_argument("--serve-creators", type=int, default=8,
                    help="serving: threads creating and retiring request state")
    ap.add_argument("--serve-depth", type=int, default=2,
                    help="serving ticks queued on the device at once (1: read each before the next)")
    ap.add_argument("--serve-blocking", type=int, default=0,
                    help="1: the library's host waits sleep instead of spinning while serving")
    ap.add_argument("--serve-streams", type=int, default=2,
                    help="streams the serving ticks take in turn (with --serve-depth >= 2 they overlap)")
    ap.add_argument("--serve-join-at", type=int, default=0,
                    help="serving: staged requests join only when at most this many run (0: at every round)")
    ap.add_argument("--serve-ctas", type=int, default=0,
                    help="serving: CTAs per SM of the batch's persistent kernels (0 = occupancy)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--no-batch", action="store_true",
                    help="default workload: skip the batched-vs-plain section")
    ap.add_argument("--no-serving", action="store_true",
                    help="default workload: skip the serving section")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--subrounds", type=int, default=4)
    ap.add_argument("--variant", choices=["plain", "balance", "revert", "balance+revert"], default="plain",
                    help="LP variant of Sec. 6: zero-gain balance moves and/or revert of negative "
                         "attributed gains")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-pool-retention", type=int, default=64 << 30,
                    help="device bytes the library's pool keeps between end-to-end steps (0: none)")
    ap.add_argument("--l2-fetch-granularity", type=int, default=0,
                    help="measurement option: the context's maximum L2 fetch granularity in bytes (0: default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    elif args.workload == "batch":
        rc = run_batch(args, world, rank, local)
    elif args.workload == "serving":
        rc = run_serving(args, world, rank, local)
    elif args.workload == "rebalance":
        rc = run_rebalance(args, world, rank, local)
    elif args.workload == "contract":
        rc = run_contract(args, world, rank, local)
    else:
        rc = run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
