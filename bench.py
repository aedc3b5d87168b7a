#!/usr/bin/env python
"""HashGraph benchmark on GB300.

Default workload (the headline line): one step = the whole hot path over one
batch of synthetic input, HashGraph-V2 build (Alg. 2) of N = 2^28 uniform
uint32 keys into V = 2^28 buckets (load factor 1), then the binned probe
(HashGraph-Probe-Standard semantics, queries grouped by bucket range so every
group probes an L2-resident slice of the table) of Q = 2^28 queries at 50%
hits.  value = (N + Q) / step time in Gkeys/s, summed over ranks (each rank
builds and probes its own table: weak scaling, no collective).  Inputs (2 GiB
per step) exceed the 129 MB L2, so no flush is needed between steps.

Other workloads (one JSON line each, same keys), chosen by --workload:
  plain    2^20 keys, 2^20 buckets, 2^20 queries (the oracle-sized case)
  (scale and plain take --dup D: keys drawn uniformly from [1 .. N/D], an
  average of D appearances per key, as in the duplicate-key experiment)
  join     Alg. 3: build 2^27 uint64 Zipf(1) keys over 2^24 values and 2^27
           uniform keys over the same values, join count and materialise
  batched  10,000 tables, log-uniform sizes scaled to a 2^30-key total, each
           probed by as many queries (50% hits), one graph launch per step
           (autotuned); compared with a host loop of plain calls
  learned  2^27 uint64 lognormal-mixture keys, learned bucket map (trained
           once, on the GPU) vs Murmur: build + binned probe of 2^27 queries

    python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload W]

Prints ONE JSON line on rank 0.  With the default workload on one GPU the
line also carries a "workloads" object: a short run (--workload-steps timed
steps after 3 warm-ups) of each other workload, with its own value, phases,
roofline and CPU baseline (--no-workloads leaves it out).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HashGraph build & probe Gkeys/s at 2^28 keys; % of HBM roofline"
UNIT = "Gkeys/s"
WORKLOADS = ("scale", "plain", "join", "batched", "learned")



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hg", "reference"], default="hg")
    ap.add_argument("--workload", choices=WORKLOADS, default="scale")
    ap.add_argument("--log2n", type=int, default=None)
    ap.add_argument("--log2v", type=int, default=None)
    ap.add_argument("--hit", type=float, default=0.5)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--e2e-slots", type=int, default=2, help="batches in flight in the end-to-end measurement")
    ap.add_argument("--standard-probe", action="store_true", help="time HashGraph-Probe-Standard instead of the binned probe")
    ap.add_argument("--algo", choices=["v2", "v1"], default="v2", help="build algorithm (Alg. 2 or Alg. 1)")
    ap.add_argument("--explicit-ids", action="store_true", help="build with a uint32 id array (+4 B read per key)")
    ap.add_argument("--dup", type=float, default=0.0,
                    help="scale/plain: keys drawn uniformly from [1 .. N/D], D appearances per key on average "
                         "(the duplicate-key experiment); 0 = distinct-looking uniform keys")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned-join", action="store_true",
                    help="learned workload: skip the learned vs murmur3 join of the key and query tables")
    ap.add_argument("--cpu-log2n", type=int, default=25, help="oracle sample size (log2 keys; 2^25 is about 10 s of CPU work)")
    ap.add_argument("--cpu-mt-log2n", type=int, default=24,
                    help="sample size of the multithreaded CPU HashGraph (log2 keys); 0 = skip it")
    ap.add_argument("--plain-steps", type=int, default=2, help="batched: timed runs of the per-table loop")
    ap.add_argument("--no-workloads", action="store_true",
                    help="headline only: skip the other workloads the default line reports under 'workloads'")
    ap.add_argument("--workload-steps", type=int, default=5, help="timed steps of each secondary workload")
    a = ap.parse_args()
    if a.log2n is None:
        a.log2n = 20 if a.workload == "plain" else 28
    return a


# --------------------------------------------------------------------------
# environment helpers
# --------------------------------------------------------------------------
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def src_digest() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1907_02900_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


# Nominal HBM3e bandwidth of a GB300 (about 8 TB/s), reported beside the
# measured copy bandwidth, which is the roofline's peak.
HBM_NOMINAL_GBS = 8000.0

# The workload the committed DRAM captures were taken on: uint32 keys with
# implicit ids, Murmur map, V = N (load 1), 50% hits, inputs beyond L2.  Other
# workloads run other kernel instantiations or other bytes per unit (8-byte
# keys, another load factor, an L2-resident table), so they get no figure.
TRAFFIC_WORKLOAD = "scale"


def recorded_traffic(kernel: str, units: int, workload: str | None = None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    by the units (keys or queries) one launch processes; None when absent,
    taken on other kernel sources, or taken on another workload."""
    if workload != TRAFFIC_WORKLOAD:
        return None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    e = t.get(kernel)
    if not e or e.get("src_digest") != src_digest():
        return None
    return int(e["bytes_per_unit"] * units)


# --------------------------------------------------------------------------
# algorithmic bytes of each kernel per launch (element granularity: every
# input read once, every output written once)
# --------------------------------------------------------------------------
PROBE_KERNELS = {"k_hist_Q", "k_colscan_Q", "k_scan_Q", "k_partition_Q", "k_probe", "k_unpermute"}


def algo_build(kb: int, n: int, V: int) -> dict:
    return {
        "k_hist": kb * n,                                  # read keys
        "k_partition_A": kb * n + (kb + 4) * n,            # read keys, write (key, id)
        "k_partition_B": 2 * (kb + 4) * n,                 # read and write (key, id)
        "k_binbuild": 2 * (kb + 4) * n + 4 * V,            # read (key, id), write CSR + offsets
    }


def algo_probe(kb: int, n: int, V: int, q: int, hit: float, binned: bool = True, positions: bool = False) -> dict:
    """positions: the probe also reads each grouped query's position (batched
    tables, whose bucket map needs it)."""
    table = 4 * (V + 1) + kb * n
    if binned:
        return {
            "k_hist_Q": kb * q,                            # read queries
            "k_partition_Q": kb * q + (kb + 4) * q,        # read queries, write (query, position)
            "k_probe": kb * q + 4 * q + (4 * q if positions else 0) + table,  # grouped queries, counts, table once
            "k_unpermute": 3 * 4 * q,                      # read (position, count), write counts
        }
    alpha = n / V
    nonempty = hit + (1.0 - hit) * (1.0 - math.exp(-alpha))
    return {"k_probe": q * (kb + 4) + q * 32 + q * 32 * nonempty}  # 32 B sectors: offsets, first key


def algo_join(kb: int, nA: int, nB: int, V: int, M: int) -> dict:
    return {
        # both key arrays, both offsets, m out, per-bucket counts out
        "k_join_merge": kb * nA + kb * nB + 8 * (V + 1) + 8 * nA + 8 * V,
        "k_join_write": (kb + 4) * (nA + nB) + 8 * (V + 1) + 8 * nA + 16 * M,  # keys + ids, offsets, m, pairs
    }


def roofline(prof: dict, algo: dict, steps: int, elapsed_ms: float, hbm: float, peak_src: str, units: dict,
             workload: str | None = None):
    """Per-kernel rates from the live CUDA-event profile.  algo and units are
    per step (all launches of the kernel in one step); achieved = bytes moved
    over the kernel's total time, i.e. per launch on average."""
    phases = {}
    for k, (ms, c) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        e = {"avg_ms": round(ms / max(c, 1), 4), "launches": c, "share": round(ms / max(elapsed_ms, 1e-9), 4)}
        if k in algo:
            gbs = algo[k] * steps / (ms * 1e-3) / 1e9
            e.update({"algo_bytes_per_launch": int(algo[k] * steps / max(c, 1)), "gbs": round(gbs, 1),
                      "frac": round(gbs / hbm, 4)})
        phases[k] = e
    cand = [k for k in prof if k in algo]
    if not cand:
        return None, phases
    dom = max(cand, key=lambda k: prof[k][0])
    ms, c = prof[dom]
    ach = algo[dom] * steps / (ms * 1e-3) / 1e9
    per_launch_units = units.get(dom, 0) * steps / max(c, 1)
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(ach / hbm, 4), "traffic": recorded_traffic(dom, per_launch_units, workload),
            "peak_source": f"hbm_gbs of {peak_src}",
            "peak_nominal": HBM_NOMINAL_GBS, "frac_nominal": round(ach / HBM_NOMINAL_GBS, 4)}
    return roof, phases


# --------------------------------------------------------------------------
class Ctx:
    """Device, ranks and the timed-region helper shared by every workload."""

    def __init__(self, args):
        import torch
        import paper_1907_02900_gb300 as hg
        self.torch, self.hg, self.args = torch, hg, args
        self.world, self.rank, self.local = dist_info()
        if self.world > 1:
            import torch.distributed as dist
            torch.cuda.set_device(self.local)
            dist.init_process_group("nccl")
        else:
            torch.cuda.set_device(0)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        from paper_1907_02900_gb300 import _build
        _build.build()
        hg.load()
        self.stream = torch.cuda.current_stream()
        peaks, src = measured_peaks()
        self.hbm, self.peak_src = float(peaks.get("hbm_gbs", 6800.0)), src

    def barrier(self):
        if self.world > 1:
            self.torch.distributed.barrier()

    def rate(self, units_local: float, elapsed_ms_local: float) -> tuple[float, float]:
        """(Gunits/s summed over ranks, slowest rank's ms)."""
        from paper_1907_02900_gb300.replicas import whole_job_rate
        r, ms = whole_job_rate(units_local, elapsed_ms_local, self.dev if self.world > 1 else None)
        return r / 1e9, ms

    def max_over_ranks(self, x: float) -> float:
        if self.world == 1:
            return x
        t = self.torch.tensor([x], device=self.dev, dtype=self.torch.float64)
        self.torch.distributed.all_reduce(t, op=self.torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def timed(self, fn, steps: int, profile: bool = True):
        """Run fn() `steps` times between CUDA events (barrier + sync on both
        sides); returns (this rank's ms, clocks, per-kernel profile)."""
        torch, hg = self.torch, self.hg
        sampler = ClockSampler(self.local) if self.rank == 0 else None
        hg.profile_reset()
        hg.profile_enable(profile)
        self.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(steps):
            fn()
        e1.record(self.stream)
        torch.cuda.synchronize()
        self.barrier()
        clocks = sampler.stop() if sampler else None
        hg.profile_enable(False)
        prof = hg.profile_read() if profile else {}
        hg.profile_reset()
        return e0.elapsed_time(e1), clocks, prof

    def line(self, workload: str, value: float, ms_per_step: float, dtype: str, config: dict, **extra) -> dict:
        a = self.args
        d = {"metric": METRIC if workload == "scale" else f"{workload}: build & probe Gkeys/s", "value": round(value, 3),
             "unit": UNIT, "n_gpus": self.world, "steps": a.steps, "warmup": a.warmup,
             "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
             "dtype": dtype, "data": "synthetic", "config": config}
        d.update(extra)
        d["gpu"] = self.torch.cuda.get_device_name(self.dev)
        return d

    def check_ws(self, ws, where: str):
        st = self.hg.workspace_status(ws)
        if st != 0:
            raise RuntimeError(f"{where}: device status {self.hg.STATUS_NAMES.get(st, st)}")


def oracle_sample(log2n: int, log2v: int, hit: float, seed: int, dup: float = 0.0):
    """Oracle (single-threaded CPU) build + probe of a bounded sample; returns (seconds, keys)."""
    import oracle
    from paper_1907_02900_gb300 import datagen as dg
    n = 1 << log2n
    V = 1 << log2v
    keys = dg.dup_keys_u32(n, dup, seed) if dup > 0 else dg.uniform_keys_u32(n, seed)
    q = dg.queries_u32(n, keys, hit, seed + 1)
    oracle.build_oracle()
    t0 = time.perf_counter()
    off, ck, _ = oracle.build(keys, V)
    oracle.probe(off, ck, q, V)
    return time.perf_counter() - t0, 2 * n


def cpu_mt_sample(log2n: int, log2v: int, hit: float, seed: int, dup: float = 0.0) -> dict:
    """The multithreaded CPU HashGraph (all host cores) on a bounded sample of
    the workload: build + probe, median of three runs after a warm-up.  Never
    raises: a failure is reported in the line instead."""
    try:
        import cpu_baseline as cmt
        from paper_1907_02900_gb300 import datagen as dg
        n, V = 1 << log2n, 1 << log2v
        keys = dg.dup_keys_u32(n, dup, seed) if dup > 0 else dg.uniform_keys_u32(n, seed)
        q = dg.queries_u32(n, keys, hit, seed + 1)
        threads = cmt.max_threads()
        off, ck, _ = cmt.build(keys[: 1 << 16], 1 << 16, threads=threads)
        cmt.probe(off, ck, 1 << 16, q[: 1 << 16], threads=threads)
        secs = []
        for _ in range(3):
            t0 = time.perf_counter()
            off, ck, _ = cmt.build(keys, V, threads=threads)
            cmt.probe(off, ck, V, q, threads=threads)
            secs.append(time.perf_counter() - t0)
        t = sorted(secs)[1]
        return {"value": 2 * n / t / 1e9, "unit": UNIT, "cores": threads, "kind": "openmp HashGraph-V2",
                "sample": f"build of 2^{log2n} uint32 keys into 2^{log2v} buckets + probe of 2^{log2n} queries "
                          f"({int(hit * 100)}% hits), median of 3: {t:.3f} s; nproc={os.cpu_count()}"}
    except Exception as e:  # the GPU line must not depend on the CPU comparison
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}


def cpu_line(secs: float, units: float, sample: str) -> dict:
    return {"value": units / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sample}, {secs:.1f} s single-threaded; nproc={os.cpu_count()}"}


# --------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    log2v_full = args.log2v if args.log2v is not None else args.log2n
    ln = min(args.cpu_log2n, args.log2n)
    lv = ln + (log2v_full - args.log2n)
    for _ in range(max(args.warmup, 0) and 1):
        oracle_sample(ln - 4, lv - 4, args.hit, 7, args.dup)
    total_s, total_keys = 0.0, 0
    for i in range(args.steps):
        s, k = oracle_sample(ln, lv, args.hit, 0x48470002 + i, args.dup)
        total_s += s
        total_keys += k
    value = total_keys / total_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"oracle sample: 2^{ln} uint32 "
                               f"{f'keys from [1 .. N/{args.dup:g}]' if args.dup > 0 else 'uniform keys'}, V=2^{lv}, probe 2^{ln} queries at "
                               f"{int(args.hit * 100)}% hits (same shape as 2^{args.log2n} keys, V=2^{log2v_full})",
                   "parallelism": "single-threaded CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"build+probe of 2^{ln} keys per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
def run_scale(c: Ctx):
    """Build + probe of one table (the headline; also the 2^20 'plain' case)."""
    torch, hg, args = c.torch, c.hg, c.args
    from paper_1907_02900_gb300 import datagen as dg
    n = 1 << args.log2n
    log2v = args.log2v if args.log2v is not None else args.log2n
    V = 1 << log2v
    q = n
    seed = dg.SEED_SCALE + 1000 * c.rank
    import paper_1907_02900_gb300.datagen_gpu as dgg
    if args.dup > 0:
        keys_h = dg.dup_keys_u32(n, args.dup, seed)
        keys_d = torch.from_numpy(keys_h.view(np.int32)).to(c.dev).view(torch.uint32)
        del keys_h
    else:   # the same numbers as datagen.uniform_keys_u32, drawn on the device
        keys_d = dgg.uniform_keys_u32(n, seed, device=c.dev)
    q_d = dgg.queries_u32(q, keys_d, args.hit, seed + 1)
    # pinned host copies for the end-to-end leg
    keys_p = torch.empty(n, dtype=torch.int32, pin_memory=True) if args.e2e_steps > 0 else None
    q_p = torch.empty(q, dtype=torch.int32, pin_memory=True) if args.e2e_steps > 0 else None
    if keys_p is not None:
        keys_p.copy_(keys_d.view(torch.int32))
        q_p.copy_(q_d.view(torch.int32))
    cfg = hg.make_config(hg.KEY_U32, V, 0, args.algo)
    ids_d = None
    if args.explicit_ids:   # a permutation-like id array: ids = position * odd constant (mod 2^32)
        ids_d = (torch.arange(n, dtype=torch.int64, device=c.dev) * 2654435761 % (1 << 32)).to(torch.int32).view(
            torch.uint32)
    ws = torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=c.dev)
    offsets = torch.empty(V + 1, dtype=torch.uint32, device=c.dev)
    ck = torch.empty(n, dtype=torch.uint32, device=c.dev)
    ci = torch.empty(n, dtype=torch.uint32, device=c.dev)
    counts = torch.empty(q, dtype=torch.uint32, device=c.dev)
    table = hg.Table(offsets, ck, ci, cfg)
    binned = not args.standard_probe
    pws = torch.empty(max(hg.probe_workspace_size(table, q), 1), dtype=torch.uint8, device=c.dev) if binned else None

    def step(kd, qd):
        hg.build_into(cfg, kd, ids_d, offsets, ck, ci, ws, c.stream)
        if binned:
            hg.probe_binned_into(table, qd, counts, pws, c.stream)
        else:
            hg.probe_into(table, qd, counts, c.stream)

    for _ in range(args.warmup):
        step(keys_d, q_d)
    torch.cuda.synchronize()
    c.check_ws(ws, "build")
    if binned:
        c.check_ws(pws, "probe")
    local_ms, clocks, prof = c.timed(lambda: step(keys_d, q_d), args.steps)
    value, elapsed_ms = c.rate((n + q) * args.steps, local_ms)
    ms_per_step = elapsed_ms / args.steps
    algo = dict(algo_build(4, n, V), **algo_probe(4, n, V, q, args.hit, binned))
    if args.explicit_ids:
        algo["k_partition_A"] += 4 * n        # the id array is read too
    if args.algo == "v1":
        for k in ("k_hist", "k_partition_A", "k_partition_B", "k_binbuild"):
            algo.pop(k)
    units = {k: (q if k in PROBE_KERNELS else n) for k in algo}
    # the committed DRAM captures hold for this shape only (sizes they were taken at)
    captured_shape = (args.log2n in (27, 28) and V == n and args.hit == 0.5 and args.dup == 0
                      and not args.explicit_ids and args.algo == "v2" and binned)
    roof, phases = roofline(prof, algo, args.steps, elapsed_ms, c.hbm, c.peak_src, units,
                            TRAFFIC_WORKLOAD if captured_shape else None)
    build_ms = sum(prof[k][0] for k in prof if k not in PROBE_KERNELS) / args.steps
    probe_ms = sum(prof[k][0] for k in prof if k in PROBE_KERNELS) / args.steps

    e2e = None
    if args.e2e_steps > 0:
        # Through the public host-buffer call (hg_build_probe_host): keys and
        # queries from pinned host memory, counts back to pinned host memory,
        # every step.  Several batches in flight on their own streams, as a
        # serving loop would run it, so one batch's copies overlap the others'
        # kernels.
        del ws, offsets, ck, ci, counts, pws, table
        slots = []
        for _ in range(args.e2e_slots):
            sl = {"stream": torch.cuda.Stream(device=c.dev),
                  "dk": torch.empty(n, dtype=torch.uint32, device=c.dev),
                  "dq": torch.empty(q, dtype=torch.uint32, device=c.dev),
                  "dc": torch.empty(q, dtype=torch.uint32, device=c.dev),
                  "table": hg.Table(torch.empty(V + 1, dtype=torch.uint32, device=c.dev),
                                    torch.empty(n, dtype=torch.uint32, device=c.dev),
                                    torch.empty(n, dtype=torch.uint32, device=c.dev), cfg),
                  "hc": torch.empty(q, dtype=torch.int32).pin_memory()}
            sl["ws"] = torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=c.dev)
            sl["pws"] = (torch.empty(hg.probe_workspace_size(sl["table"], q), dtype=torch.uint8, device=c.dev)
                         if binned else None)
            slots.append(sl)

        def host_step(i):
            sl = slots[i % args.e2e_slots]
            hg.build_probe_host(cfg, keys_p, q_p, sl["hc"], sl["dk"], sl["dq"], sl["dc"], sl["table"], sl["ws"],
                                sl["pws"], stream=sl["stream"])

        for i in range(args.e2e_slots):   # warm-up of every slot
            host_step(i)
        torch.cuda.synchronize()
        # the host link's own copy rates on this machine (pinned buffers, one copy
        # each way of the keys), which bound the end-to-end rate
        link = {}
        for name, dst, src in (("h2d_gbs", slots[0]["dk"].view(torch.int32), keys_p),
                               ("d2h_gbs", keys_p, slots[0]["dk"].view(torch.int32))):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(c.stream)
            dst.copy_(src, non_blocking=True)
            e1.record(c.stream)
            torch.cuda.synchronize()
            link[name] = round(4 * n / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1)
        c.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(c.stream)
        for sl in slots:
            sl["stream"].wait_stream(c.stream)
        for i in range(args.e2e_steps):
            host_step(i)
        for sl in slots:
            c.stream.wait_stream(sl["stream"])
        e1.record(c.stream)
        torch.cuda.synchronize()
        c.barrier()
        e2e_value, _ = c.rate((n + q) * args.e2e_steps, e0.elapsed_time(e1))
        last = slots[(args.e2e_steps - 1) % args.e2e_slots]
        ok = bool(np.array_equal(last["hc"].numpy().view(np.uint32), last["dc"].cpu().numpy()))
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": 4 * (n + q), "d2h_bytes_per_step": 4 * q,
               "call": f"hg_build_probe_host, pinned host buffers, {args.e2e_slots} batches in flight",
               "counts_returned": ok, "host_link": link}
        del slots

    # Duplicate keys come from [1 .. N/D] as raw values, so a miss query (a
    # scrambled value from the upper half of the domain) can equal one of
    # them with probability about (N/D) / 2^32: the hit rate is then slightly
    # above the requested one.
    key_kind = f"keys from [1 .. N/{args.dup:g}]" if args.dup > 0 else "uniform keys"
    cpu = None
    if c.rank == 0 and c.world == 1 and not args.no_cpu_baseline:
        ln = min(args.cpu_log2n, args.log2n)
        lv = ln + (log2v - args.log2n)
        secs, done = oracle_sample(ln, lv, args.hit, seed + 7, args.dup)
        cpu = cpu_line(secs, done, f"oracle build of 2^{ln} uint32 {key_kind} into 2^{lv} buckets + probe of "
                                   f"2^{ln} queries ({int(args.hit * 100)}% hits)")
    cpu_mt = None
    if c.rank == 0 and c.world == 1 and not args.no_cpu_baseline and args.cpu_mt_log2n > 0:
        ln = min(args.cpu_mt_log2n, args.log2n)
        cpu_mt = cpu_mt_sample(ln, ln + (log2v - args.log2n), args.hit, seed + 9, args.dup)
    algo_name = "HashGraph-V2" if args.algo == "v2" else "HashGraph-V1"
    ids_name = "explicit uint32 ids" if args.explicit_ids else "implicit ids"
    config = {"workload": f"{algo_name} build of 2^{args.log2n} uint32 {key_kind} ({ids_name}) into 2^{log2v} "
                          f"buckets (murmur3) + {'binned probe' if binned else 'Probe-Standard'} of 2^{args.log2n} "
                          f"queries at {int(args.hit * 100)}% hits, per GPU",
              "global_batch": c.world * (n + q),
              "l2": "inputs (8 B per key and query) exceed L2; no flush" if n >= 1 << 24 else
                    "inputs fit in L2 (small case); no flush",
              "parallelism": f"replicas x{c.world} (independent tables per GPU)"}
    # the whole step against its minimum traffic: keys read, CSR + offsets written,
    # queries read, counts written, the table read once
    min_bytes = 4 * n + 8 * n + 4 * (V + 1) + 4 * q + 4 * q + (4 * (V + 1) + 4 * n)
    return c.line("scale" if args.workload == "scale" else args.workload, value, ms_per_step, "u32", config,
                  build_gkeys_s=round(n / (build_ms * 1e-3) / 1e9, 3) if build_ms else None,
                  probe_gkeys_s=round(q / (probe_ms * 1e-3) / 1e9, 3) if probe_ms else None,
                  end_to_end_min_bytes_frac=round(min_bytes / (ms_per_step * 1e-3) / 1e9 / c.hbm, 4),
                  probe="binned" if binned else "standard", roofline=roof, phases=phases, cpu_baseline=cpu,
                  cpu_mt_baseline=cpu_mt,
                  e2e=e2e, gpu_launches=sum(v[1] for v in prof.values()), clocks=clocks)


def run_join(c: Ctx):
    torch, hg, args = c.torch, c.hg, c.args
    from paper_1907_02900_gb300 import datagen as dg
    n = 1 << 27
    distinct = 1 << 24
    V = 1 << 27
    seed = dg.SEED_JOIN + 1000 * c.rank
    a_h = dg.zipf_keys_u64(n, distinct, seed, 1.0)
    b_h = dg.uniform_domain_keys_u64(n, distinct, seed + 1)
    a_d = torch.from_numpy(a_h.view(np.int64)).to(c.dev).view(torch.uint64)
    b_d = torch.from_numpy(b_h.view(np.int64)).to(c.dev).view(torch.uint64)
    cfg = hg.make_config(hg.KEY_U64, V, 0, "v2")
    ws = torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=c.dev)

    def alloc_table():
        return hg.Table(torch.empty(V + 1, dtype=torch.uint32, device=c.dev),
                        torch.empty(n, dtype=torch.uint64, device=c.dev),
                        torch.empty(n, dtype=torch.uint32, device=c.dev), cfg)

    tA, tB = alloc_table(), alloc_table()
    jws = torch.empty(hg.join_workspace_size(cfg, n, n), dtype=torch.uint8, device=c.dev)
    total = torch.empty(1, dtype=torch.int64, device=c.dev)
    hg.build_into(cfg, a_d, None, tA.offsets, tA.keys, tA.ids, ws, c.stream)
    hg.build_into(cfg, b_d, None, tB.offsets, tB.keys, tB.ids, ws, c.stream)
    hg.join_count_into(tA, tB, total, None, jws, c.stream)
    M = int(total.item())
    out_a = torch.empty(max(M, 1), dtype=torch.int64, device=c.dev)
    out_b = torch.empty(max(M, 1), dtype=torch.int64, device=c.dev)

    def step():
        hg.build_into(cfg, a_d, None, tA.offsets, tA.keys, tA.ids, ws, c.stream)
        hg.build_into(cfg, b_d, None, tB.offsets, tB.keys, tB.ids, ws, c.stream)
        hg.join_count_into(tA, tB, total, None, jws, c.stream)
        # the pairs are written from the per-edge counts the count pass left in jws
        hg.join_materialize_into(tA, tB, out_a, out_b, total, jws, c.stream, after_count=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    c.check_ws(ws, "build")
    c.check_ws(jws, "join")
    local_ms, clocks, prof = c.timed(step, args.steps)
    value, elapsed_ms = c.rate(2 * n * args.steps, local_ms)
    ms = elapsed_ms / args.steps
    # two builds per step
    algo = {k: 2 * v for k, v in algo_build(8, n, V).items()}
    algo.update(algo_join(8, n, n, V, M))
    units = {k: 2 * n if k in algo_build(8, 1, 1) or k == "k_join_merge" else n for k in algo}
    roof, phases = roofline(prof, algo, args.steps, elapsed_ms, c.hbm, c.peak_src, units)
    join_ms = sum(prof[k][0] for k in prof if k.startswith("k_join") or k.startswith("k_scan")) / args.steps
    cpu = None
    if c.rank == 0 and c.world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build_oracle()
        m = 1 << 21
        sa = dg.zipf_keys_u64(m, distinct >> 6, seed + 2, 1.0)
        sb = dg.uniform_domain_keys_u64(m, distinct >> 6, seed + 3)
        t0 = time.perf_counter()
        offA, kA, iA = oracle.build(sa, m)
        offB, kB, iB = oracle.build(sb, m)
        oracle.join_count(offA, kA, offB, kB, m)
        secs = time.perf_counter() - t0
        cpu = cpu_line(secs, 2 * m, f"oracle builds of 2 x 2^21 uint64 keys (same shape, 2^18 distinct) + join count")
    config = {"workload": "Alg. 3 join: build 2^27 uint64 Zipf(1.0) keys over 2^24 values and 2^27 uniform keys over "
                          "the same values into 2^27 buckets each (V2), join count + materialise int64 pairs",
              "global_batch": c.world * 2 * n, "l2": "inputs exceed L2; no flush",
              "parallelism": f"replicas x{c.world}", "pairs": M}
    return c.line("join", value, ms, "u64", config, pairs_per_s=round(c.rate(M * args.steps, local_ms)[0], 3),
                  join_ms=round(join_ms, 3), roofline=roof, phases=phases, cpu_baseline=cpu, e2e=None,
                  gpu_launches=sum(v[1] for v in prof.values()), clocks=clocks)


def run_batched(c: Ctx):
    torch, hg, args = c.torch, c.hg, c.args
    from paper_1907_02900_gb300 import datagen as dg
    import paper_1907_02900_gb300.datagen_gpu as dgg
    T = 10_000
    sizes = dg.batched_sizes(T, dg.SEED_BATCH, total=(1 << 30) - 4 * T)
    qsizes = sizes.copy()
    plan = hg.BatchPlan(sizes, qsizes, seed=dg.SEED_BATCH)
    b = plan.alloc(c.dev)
    dgg.fill_batch(plan, b, key_seed=dg.SEED_BATCH + 1 + c.rank, query_seed=dg.SEED_BATCH + 2 + c.rank,
                   hit_rate=args.hit)
    t0 = time.perf_counter()
    tuned = plan.autotune(b, reps=2)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        plan.run(b)
    torch.cuda.synchronize()
    c.check_ws(b["ws"], "batch")
    units = int(sizes.sum() + qsizes.sum())
    local_ms, clocks, _ = c.timed(lambda: plan.run(b), args.steps, profile=False)
    value, elapsed_ms = c.rate(units * args.steps, local_ms)
    ms = elapsed_ms / args.steps
    # per-kernel breakdown from one eager (uncaptured) run of the same sequence
    eager_ms, _, prof = c.timed(lambda: plan.run_eager(b), 1)
    n, q, V = int(plan.total_keys), int(plan.total_queries), int(plan.total_offsets - 1)
    algo = dict(algo_build(4, n, V), **algo_probe(4, n, V, q, args.hit, True, positions=True))
    algo_total = sum(algo.values())
    kunits = {k: (q if k in PROBE_KERNELS else n) for k in algo}
    roof_k, phases = roofline(prof, algo, 1, eager_ms, c.hbm, c.peak_src, kunits)
    # per-kernel launch totals sum the waves; the whole graph against all kernels' bytes
    ach = algo_total / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "whole batch (one graph launch)", "achieved": round(ach, 1), "peak": c.hbm,
            "unit": "GB/s", "frac": round(ach / c.hbm, 4), "traffic": None, "peak_source": f"hbm_gbs of {c.peak_src}",
            "dominant_kernel": roof_k}
    plain_ms = None
    if args.plain_steps > 0:
        plan.run_plain(b)
        torch.cuda.synchronize()
        pm, _, _ = c.timed(lambda: plan.run_plain(b), args.plain_steps, profile=False)
        plain_ms = c.max_over_ranks(pm) / args.plain_steps
        plan.run(b)
    cpu = None
    if c.rank == 0 and c.world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build_oracle()
        ub = np.concatenate([[0], np.cumsum(sizes)])
        rng = np.random.default_rng(1)
        pick = rng.choice(T, 200, replace=False)
        done, secs = 0, 0.0
        for t in pick:
            kt = dg.uniform_keys_u32(int(sizes[t]), dg.SEED_BATCH + 1, start=int(ub[t]))
            qt = dg.batched_table_queries_u32(int(qsizes[t]), int(ub[t]), kt, args.hit, dg.SEED_BATCH + 2)
            s0 = time.perf_counter()
            off, ck, _ = oracle.build(kt, int(sizes[t]), seed=dg.SEED_BATCH)
            oracle.probe(off, ck, qt, int(sizes[t]), seed=dg.SEED_BATCH)
            secs += time.perf_counter() - s0
            done += len(kt) + len(qt)
        cpu = cpu_line(secs, done, f"oracle build + probe of 200 random tables of the batch ({done} keys+queries)")
    config = {"workload": f"{T} tables, log-uniform sizes scaled to {int(sizes.sum())} uint32 keys in total "
                          f"({int(sizes.min())}..{int(sizes.max())} per table), V_t = n_t, as many queries at "
                          f"{int(args.hit * 100)}% hits; build + binned probe of every table, one CUDA graph launch",
              "global_batch": c.world * units, "l2": "inputs exceed L2; no flush",
              "parallelism": f"replicas x{c.world}", "autotuned": tuned, "autotune_s": round(tune_s, 2),
              "waves": plan.config()["waves"]}
    return c.line("batched", value, ms, "u32", config,
                  plain_loop_gkeys_s=round(c.world * units / (plain_ms * 1e-3) / 1e9, 3) if plain_ms else None,
                  speedup_vs_plain_loop=round(plain_ms / ms, 2) if plain_ms else None,
                  roofline=roof, phases=phases, cpu_baseline=cpu, e2e=None,
                  gpu_launches=sum(v[1] for v in prof.values()) * args.steps, clocks=clocks)


def learned_joins(c: Ctx, keys_d, q_d, V: int, model) -> dict:
    """Alg. 3 join of the key table with a table of the queries, both built
    with the learned map and both with murmur3: count + materialise, timed
    alone (the tables are built before the timed region).  The pair sets
    must be equal (their order follows each map's buckets)."""
    torch, hg, args = c.torch, c.hg, c.args
    out = {}
    pairs = {}
    for name, mdl in (("learned", model), ("murmur", None)):
        cfg = hg.make_config(hg.KEY_U64, V, 0, "v2", model=mdl)
        tabs = []
        for src in (keys_d, q_d):
            n = src.numel()
            ws = torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=c.dev)
            t = hg.Table(torch.empty(V + 1, dtype=torch.uint32, device=c.dev),
                         torch.empty(n, dtype=torch.uint64, device=c.dev),
                         torch.empty(n, dtype=torch.uint32, device=c.dev), cfg, model=mdl)
            hg.build_into(cfg, src, None, t.offsets, t.keys, t.ids, ws, c.stream)
            c.torch.cuda.synchronize()
            c.check_ws(ws, name + " join build")
            del ws
            tabs.append(t)
        tA, tB = tabs
        jws = torch.empty(hg.join_workspace_size(cfg, tA.keys.numel(), tB.keys.numel()), dtype=torch.uint8,
                          device=c.dev)
        total = torch.empty(1, dtype=torch.int64, device=c.dev)
        hg.join_count_into(tA, tB, total, None, jws, c.stream)
        M = int(total.item())
        oa = torch.empty(max(M, 1), dtype=torch.int64, device=c.dev)
        ob = torch.empty(max(M, 1), dtype=torch.int64, device=c.dev)

        def step():
            hg.join_count_into(tA, tB, total, None, jws, c.stream)
            hg.join_materialize_into(tA, tB, oa, ob, total, jws, c.stream, after_count=True)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        c.check_ws(jws, name + " join")
        el, _, prof = c.timed(step, args.steps)
        ms = el / args.steps
        pairs[name] = torch.sort((oa[:M] << 32) | ob[:M])[0]
        out[name + "_ms"] = round(ms, 4)
        out[name + "_phases_avg_ms"] = {k: round(v[0] / max(v[1], 1), 4) for k, v in prof.items()}
        out["pairs"] = M
        del tabs, tA, tB, jws, oa, ob
    out["learned_vs_murmur"] = round(out["murmur_ms"] / out["learned_ms"], 3)
    out["identical_pairs"] = bool(torch.equal(pairs["learned"], pairs["murmur"]))
    out["workload"] = ("join of the key table with a table of the 2^27 queries (V = 2^27 each), count + "
                       "materialise; tables built before the timed region")
    return out


def run_learned(c: Ctx):
    torch, hg, args = c.torch, c.hg, c.args
    from paper_1907_02900_gb300 import datagen as dg
    n = 1 << 27
    V = 1 << 27
    q = n
    seed = dg.SEED_LEARNED + 1000 * c.rank
    keys_h = dg.lognormal_mixture_u64(n, seed)
    q_h = dg.queries_u64(q, keys_h, args.hit, seed + 1)
    keys_d = torch.from_numpy(keys_h.view(np.int64)).to(c.dev).view(torch.uint64)
    q_d = torch.from_numpy(q_h.view(np.int64)).to(c.dev).view(torch.uint64)
    del q_h
    # training: once per key set, timed on its own (after one untimed call
    # that loads the training kernels)
    hg.learned_train(keys_d, V)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(c.stream)
    model, diag = hg.learned_train(keys_d, V)
    t1.record(c.stream)
    torch.cuda.synchronize()
    train_ms = t0.elapsed_time(t1)
    chosen, rep = hg.choose_map(keys_d, V, model)

    def setup(mdl):
        cfg = hg.make_config(hg.KEY_U64, V, 0, "v2", model=mdl)
        ws = torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=c.dev)
        t = hg.Table(torch.empty(V + 1, dtype=torch.uint32, device=c.dev),
                     torch.empty(n, dtype=torch.uint64, device=c.dev),
                     torch.empty(n, dtype=torch.uint32, device=c.dev), cfg, model=mdl)
        pws = torch.empty(hg.probe_workspace_size(t, q), dtype=torch.uint8, device=c.dev)
        counts = torch.empty(q, dtype=torch.uint32, device=c.dev)

        def step():
            hg.build_into(cfg, keys_d, None, t.offsets, t.keys, t.ids, ws, c.stream)
            hg.probe_binned_into(t, q_d, counts, pws, c.stream)
        return step, ws, pws, counts

    res = {}
    for name, mdl in (("learned", model), ("murmur", None)):
        step, ws, pws, counts = setup(mdl)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        c.check_ws(ws, name)
        c.check_ws(pws, name)
        el, clocks, prof = c.timed(step, args.steps)
        res[name] = (el, clocks, prof, counts.clone())
        del ws, pws
    same_counts = bool(torch.equal(res["learned"][3], res["murmur"][3]))
    joins = learned_joins(c, keys_d, q_d, V, model) if not args.no_learned_join else None
    el, clocks, prof, _ = res["learned"]
    value, el_max = c.rate((n + q) * args.steps, el)
    ms = el_max / args.steps
    murmur_value, _ = c.rate((n + q) * args.steps, res["murmur"][0])
    algo = dict(algo_build(8, n, V), **algo_probe(8, n, V, q, args.hit, True))
    units = {k: (q if k in PROBE_KERNELS else n) for k in algo}
    roof, phases = roofline(prof, algo, args.steps, el, c.hbm, c.peak_src, units)
    cpu = None
    if c.rank == 0 and c.world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build_oracle()
        m = 1 << 21
        blob = model.cpu().numpy().view(np.uint8)
        ks = keys_h[:m]
        qs = dg.queries_u64(m, ks, args.hit, seed + 5)
        s0 = time.perf_counter()
        off, ck, _ = oracle.build(ks, V, model=blob)
        oracle.probe(off, ck, qs, V, model=blob)
        secs = time.perf_counter() - s0
        cpu = cpu_line(secs, 2 * m, "oracle build + probe of 2^21 of the keys with the GPU-trained learned map")
    config = {"workload": "2^27 uint64 keys, mixture of 64 lognormals (sigma 0.5..2) + 10% uniform, V = 2^27, "
                          "learned piecewise-linear CDF map (1 root + 1024 leaves, trained on a 1% sample on the GPU) "
                          "vs murmur3; V2 build + binned probe of 2^27 queries at 50% hits",
              "global_batch": c.world * (n + q), "l2": "inputs exceed L2; no flush",
              "parallelism": f"replicas x{c.world}"}
    _, _, mprof, _ = res["murmur"]
    murmur_phases = {k: round(v[0] / max(v[1], 1), 4) for k, v in sorted(mprof.items(), key=lambda kv: -kv[1][0])}
    return c.line("learned", value, ms, "u64", config, murmur_gkeys_s=round(murmur_value, 3),
                  murmur_phases_avg_ms=murmur_phases,
                  learned_vs_murmur=round(value / murmur_value, 3), identical_counts=same_counts,
                  train_ms=round(train_ms, 2), loss_before=diag["loss_before"], loss_after=diag["loss_after"],
                  bucket_stats=rep, fallback_to_murmur=not rep["kept"], join=joins, roofline=roof, phases=phases,
                  cpu_baseline=cpu, e2e=None, gpu_launches=sum(v[1] for v in prof.values()), clocks=clocks)


RUNNERS = {"scale": run_scale, "plain": run_scale, "join": run_join, "batched": run_batched, "learned": run_learned}


def run_secondary(c: Ctx) -> dict:
    """The other workloads, each a short run of its own (warm-up, timed
    steps, CPU baseline), reported beside the headline."""
    import copy
    out = {}
    base = c.args
    for name in ("plain", "join", "batched", "learned"):
        a = copy.copy(base)
        a.workload = name
        a.steps = max(1, base.workload_steps)
        a.warmup = max(3, min(base.warmup, 3))
        a.log2n = 20 if name == "plain" else 28
        a.log2v = None
        a.dup = 0.0
        a.e2e_steps = 0
        a.plain_steps = 1
        c.args = a
        try:
            t0 = time.perf_counter()
            d = RUNNERS[name](c)
            d["wall_s"] = round(time.perf_counter() - t0, 1)
            for k in ("gpu", "n_gpus", "vs_baseline", "data", "higher_is_better"):
                d.pop(k, None)
            out[name] = d
        except Exception as e:   # a secondary workload must not take the headline down
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        finally:
            c.args = base
            c.torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    c = Ctx(args)
    line = RUNNERS[args.workload](c)
    if args.workload == "scale" and not args.no_workloads and c.world == 1:
        line["workloads"] = run_secondary(c)
    if c.rank == 0:
        print(json.dumps(line), flush=True)
    if c.world > 1:
        c.torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
