#!/usr/bin/env python
"""HashGraph benchmark on GB300: build (V2) + probe throughput at 2^28 keys.

One step = one pass of the hot path over one batch of synthetic input:
HashGraph-V2 build of N = 2^28 uint32 keys into V = 2^28 buckets (load
factor 1), then HashGraph-Probe-Standard of Q = 2^28 queries (50% hits).
value = (N + Q) / step time, in Gkeys/s, summed over ranks (each rank builds
and probes its own independent table: weak scaling, no collective in the data
path).  Inputs (1 GiB of keys, 1 GiB of queries) exceed the 129 MB L2, so no
flush is needed between steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line on rank 0.
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hg", "reference"], default="hg")
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--log2v", type=int, default=None)
    ap.add_argument("--hit", type=float, default=0.5)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--standard-probe", action="store_true", help="time HashGraph-Probe-Standard instead of the binned probe")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-log2n", type=int, default=22, help="oracle sample size (log2 keys)")
    return ap.parse_args()


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


def recorded_traffic(kernel: str, n: int, V: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to this workload; None when absent or taken on other kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    e = t.get(kernel)
    if not e or e.get("src_digest") != src_digest():
        return None
    return e["bytes_per_key"] * n


# --------------------------------------------------------------------------
# algorithmic bytes of each kernel (per launch) for the uint32 workload
# --------------------------------------------------------------------------
PROBE_KERNELS = {"k_hist_Q", "k_colscan_Q", "k_scan_Q", "k_partition_Q", "k_probe", "k_unpermute"}


def algorithmic_bytes(kb: int, n: int, V: int, q: int, hit: float, binned: bool = True) -> dict:
    """Bytes each kernel must move per launch (reads + writes of its inputs and
    outputs at element granularity; the standard probe at 32-byte-sector
    granularity for its random reads)."""
    alpha = n / V
    nonempty = hit + (1.0 - hit) * (1.0 - math.exp(-alpha))
    table = 4 * (V + 1) + kb * n
    out = {
        "k_hist": kb * n,                                  # read keys
        "k_partition_A": kb * n + (kb + 4) * n,            # read keys, write (key, id)
        "k_partition_B": 2 * (kb + 4) * n,                 # read and write (key, id)
        "k_binbuild": 2 * (kb + 4) * n + 4 * V,            # read (key, id), write CSR + offsets
    }
    if binned:
        out.update({
            "k_hist_Q": kb * q,                            # read queries
            "k_partition_Q": kb * q + (kb + 4) * q,        # read queries, write (query, position)
            "k_probe": kb * q + 4 * q + table,             # read grouped queries, write counts, table once
            "k_unpermute": 3 * 4 * q,                      # read (position, count), write counts
        })
    else:
        out["k_probe"] = q * (kb + 4) + q * 32 + q * 32 * nonempty  # 32 B sectors: offsets, first key
    return out


def oracle_sample(log2n: int, log2v: int, hit: float, seed: int):
    """Oracle (single-threaded CPU) build + probe of a bounded sample; returns seconds."""
    import oracle
    from paper_1907_02900_gb300 import datagen as dg
    n = 1 << log2n
    V = 1 << log2v
    keys = dg.uniform_keys_u32(n, seed)
    q = dg.queries_u32(n, keys, hit, seed + 1)
    oracle.build_oracle()
    t0 = time.perf_counter()
    off, ck, _ = oracle.build(keys, V)
    oracle.probe(off, ck, q, V)
    return time.perf_counter() - t0, 2 * n


# --------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    log2v_full = args.log2v if args.log2v is not None else args.log2n
    ln = args.cpu_log2n
    lv = ln + (log2v_full - args.log2n)
    for _ in range(max(args.warmup, 0) and 1):
        oracle_sample(ln - 4, lv - 4, args.hit, 7)
    total_s, total_keys = 0.0, 0
    for i in range(args.steps):
        s, k = oracle_sample(ln, lv, args.hit, 0x48470002 + i)
        total_s += s
        total_keys += k
    value = total_keys / total_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"oracle sample: 2^{ln} uint32 uniform keys, V=2^{lv}, probe 2^{ln} queries at "
                               f"{int(args.hit * 100)}% hits (same shape as 2^{args.log2n} keys, V=2^{log2v_full})",
                   "parallelism": "single-threaded CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"build+probe of 2^{ln} keys per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_hg(args):
    import torch
    import paper_1907_02900_gb300 as hg
    from paper_1907_02900_gb300 import datagen as dg

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1907_02900_gb300 import _build
    _build.build()
    hg.load()

    n = 1 << args.log2n
    log2v = args.log2v if args.log2v is not None else args.log2n
    V = 1 << log2v
    q = n
    seed = dg.SEED_SCALE + 1000 * rank
    keys_h = dg.uniform_keys_u32(n, seed)
    q_h = dg.queries_u32(q, keys_h, args.hit, seed + 1)

    def pinned(a):
        t = torch.from_numpy(a.view(np.int32)).pin_memory()
        return t

    keys_p, q_p = pinned(keys_h), pinned(q_h)
    del keys_h, q_h
    keys_d = keys_p.to(dev).view(torch.uint32)
    q_d = q_p.to(dev).view(torch.uint32)
    cfg = hg.make_config(hg.KEY_U32, V, 0, "v2")
    ws_bytes = hg.build_workspace_size(cfg, n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    offsets = torch.empty(V + 1, dtype=torch.uint32, device=dev)
    ck = torch.empty(n, dtype=torch.uint32, device=dev)
    ci = torch.empty(n, dtype=torch.uint32, device=dev)
    counts = torch.empty(q, dtype=torch.uint32, device=dev)
    table = hg.Table(offsets, ck, ci, cfg)
    stream = torch.cuda.current_stream()
    binned = not args.standard_probe
    pws = torch.empty(max(hg.probe_workspace_size(table, q), 1), dtype=torch.uint8, device=dev) if binned else None

    def step(kd, qd):
        hg.build_into(cfg, kd, None, offsets, ck, ci, ws, stream)
        if binned:
            hg.probe_binned_into(table, qd, counts, pws, stream)
        else:
            hg.probe_into(table, qd, counts, stream)

    for _ in range(args.warmup):
        step(keys_d, q_d)
    torch.cuda.synchronize()
    st = hg.workspace_status(ws)
    if st != 0:
        raise RuntimeError(f"device status after warm-up: {hg.STATUS_NAMES.get(st, st)}")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    sampler = ClockSampler(local) if rank == 0 else None
    hg.profile_reset()
    hg.profile_enable(True)
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(keys_d, q_d)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    hg.profile_enable(False)
    prof = hg.profile_read()
    hg.profile_reset()
    elapsed_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    value = world * (n + q) * args.steps / (elapsed_ms * 1e-3) / 1e9
    launches = sum(c for _, c in prof.values())

    # per-kernel breakdown and the dominant kernel's roofline
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    algo = algorithmic_bytes(4, n, V, q, args.hit, binned)
    phases = {}
    for k, (ms, c) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        avg = ms / max(c, 1)
        e = {"avg_ms": round(avg, 4), "launches": c, "share": round(ms / max(elapsed_ms, 1e-9), 4)}
        if k in algo:
            gbs = algo[k] / (avg * 1e-3) / 1e9
            e.update({"algo_bytes": int(algo[k]), "gbs": round(gbs, 1), "frac": round(gbs / hbm, 4)})
        phases[k] = e
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    roof = None
    if dom:
        avg = prof[dom][0] / prof[dom][1]
        b = algo.get(dom)
        ach = b / (avg * 1e-3) / 1e9 if b else None
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1) if ach else None, "peak": hbm,
                "unit": "GB/s", "frac": round(ach / hbm, 4) if ach else None,
                "traffic": recorded_traffic(dom, n, V), "peak_source": f"hbm_gbs of {peak_src}"}
    build_ms = sum(prof[k][0] for k in prof if k not in PROBE_KERNELS) / args.steps
    probe_ms = sum(prof[k][0] for k in prof if k in PROBE_KERNELS) / args.steps

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        counts_h = torch.empty(q, dtype=torch.int32).pin_memory()
        kd2 = torch.empty(n, dtype=torch.int32, device=dev)
        qd2 = torch.empty(q, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.e2e_steps):
            kd2.copy_(keys_p, non_blocking=True)
            qd2.copy_(q_p, non_blocking=True)
            step(kd2.view(torch.uint32), qd2.view(torch.uint32))
            counts_h.copy_(counts.view(torch.int32), non_blocking=True)
        a1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = a0.elapsed_time(a1)
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": world * (n + q) * args.e2e_steps / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 4 * (n + q), "d2h_bytes_per_step": 4 * q}
        del kd2, qd2

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ln = args.cpu_log2n
        lv = ln + (log2v - args.log2n)
        secs, keys_done = oracle_sample(ln, lv, args.hit, seed + 7)
        cpu = {"value": keys_done / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"single-threaded oracle build of 2^{ln} uint32 keys into 2^{lv} buckets + probe of "
                         f"2^{ln} queries ({int(args.hit * 100)}% hits), {secs:.1f} s; nproc={os.cpu_count()}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"HashGraph-V2 build of 2^{args.log2n} uniform uint32 keys (implicit ids) into "
                                   f"2^{log2v} buckets (murmur3) + Probe-Standard of 2^{args.log2n} queries at "
                                   f"{int(args.hit * 100)}% hits, per GPU",
                       "global_batch": world * (n + q), "l2": "inputs (2 GiB per step) exceed L2; no flush",
                       "parallelism": f"replicas x{world} (independent tables per GPU)"},
            "build_gkeys_s": round(n / (build_ms * 1e-3) / 1e9, 3) if build_ms else None,
            "probe_gkeys_s": round(q / (probe_ms * 1e-3) / 1e9, 3) if probe_ms else None,
            # the whole step against its minimum traffic: build 4N read + 8N CSR + 4V offsets written,
            # probe 4Q read + 4Q written + the table read once
            "end_to_end_min_bytes_frac": round((16 * n + 4 * V + 8 * q + 4 * (V + 1) + 4 * n)
                                               / (ms_per_step * 1e-3) / 1e9 / hbm, 4),
            "probe": "binned" if binned else "standard",
            "roofline": roof, "phases": phases, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "gpu": torch.cuda.get_device_name(dev),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_hg(args)


if __name__ == "__main__":
    main()
