#!/usr/bin/env python3
"""Benchmark of the GB300 parallel in-place merge (one JSON line on rank 0).

Default workload: one stable in-place merge of int32 keys, L_A = L_B = 2^28, each run
sorted uniform values in [0, 2^31), one contiguous buffer A|B (2 GiB, larger than L2).
A step is one ipm_merge_inplace call (early exit + split + exchange levels + pair
merge).  The merge destroys its input, so before each step the buffer is restored from a
pristine device copy outside the timed interval; each step is timed with CUDA events on
the launching stream and the K step times are summed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c2-int32-uniform|c2-int32-dup16|...]

N > 1 (torchrun): the merge does not shard (a single merge needs an all-to-all that
would defeat "in place"), so every rank merges its own replica; value = all ranks' keys
/ the slowest rank's time, scaling "weak".  --impl reference times the CPU oracle (the
plain sequential merge) on a bounded sample of the same workload on host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "merged GKeys/s and % of HBM roofline: plain vs batched vs learned-split"
UNIT = "GKeys/s"

# name -> (dist, dtype, L_A, L_B, description)
WORKLOADS = {
    "c2-int32-uniform": ("uniform", "int32", 1 << 28, 1 << 28,
                         "single in-place stable merge, int32 keys, L_A=L_B=2^28, uniform "
                         "[0,2^31), one contiguous buffer A|B"),
    "c2-int32-dup16": ("dup16", "int32", 1 << 28, 1 << 28,
                       "int32 L_A=L_B=2^28, heavy duplicates U{0..15}"),
    "c2-int32-alternation": ("alternation", "int32", 1 << 28, 1 << 28,
                             "int32 L_A=L_B=2^28, A[i]=2i, B[j]=2j+1"),
    "c2-int32-unbalanced": ("uniform", "int32", 1 << 29, 1 << 20,
                            "int32 L_A=2^29, L_B=2^20, uniform"),
    "c2-uint64-uniform": ("uniform", "uint64", 1 << 28, 1 << 28,
                          "uint64 L_A=L_B=2^28, uniform [0,2^64)"),
    "c1-int32-uniform": ("uniform", "int32", 1 << 20, 1 << 20,
                         "int32 L_A=L_B=2^20, uniform (L2-resident, 8 MiB)"),
    "c2s-int32-uniform": ("uniform", "int32", 1 << 25, 1 << 25,
                          "int32 L_A=L_B=2^25, uniform (reduced c2 for profiling; 256 MiB)"),
}
NP_DT = {"int32": np.int32, "uint32": np.uint32, "uint64": np.uint64, "float32": np.float32}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c2-int32-uniform", choices=sorted(WORKLOADS))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""
    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and f[1] != self.uuid:
                continue
            rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def gpu_uuid(torch):
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ------------------------------------------------------------------ accounting

def method_bytes(n: int, w: int) -> dict:
    """Algorithmic bytes of the pair merge (every key read and written once) and of an
    out-of-place merge; the exchange's bytes come from the library after a run."""
    return {"exchange": 0, "merge": 2 * n * w, "total": 2 * n * w, "min": 2 * n * w}


# ------------------------------------------------------------------ reference arm

def cpu_oracle_timing(wl, budget_s: float = 10.0, steps: int | None = None,
                      warmup: int = 0):
    """The oracle's plain sequential merge on a 2^24+2^24-key sample of the workload
    (same generator), single thread.  Returns (GKeys/s, sample description, reps)."""
    import oracle
    import workloads

    dist, dt, la, lb, _ = wl
    scale = max(1, (la + lb) // (1 << 25))
    sa, sb = max(1, la // scale), max(1, lb // scale)
    a, b = workloads.make_pair(dist, NP_DT[dt], sa, sb, seed=0)
    oracle.merge(a[:1024], b[:1024])
    for _ in range(warmup):
        oracle.merge(a, b)
    times = []
    t_end = time.perf_counter() + budget_s
    while True:
        t0 = time.perf_counter()
        oracle.merge(a, b)
        times.append(time.perf_counter() - t0)
        if steps is not None:
            if len(times) >= steps:
                break
        elif time.perf_counter() > t_end:
            break
    tot = sum(times)
    sample = (f"oracle two-pointer merge on L_A={sa}, L_B={sb} keys of the same generator "
              f"(1/{scale} of the workload), {len(times)} reps, 1 thread")
    return (sa + sb) * len(times) / tot / 1e9, sample, len(times), tot


def run_reference(args, rank, world):
    wl = WORKLOADS[args.workload]
    if rank != 0:
        return
    t0 = time.perf_counter()
    v, sample, reps, tot = cpu_oracle_timing(wl, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot / reps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": wl[1], "data": "synthetic",
        "config": {"workload": args.workload, "description": wl[4]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t0,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world):
    import torch

    import paper_2005_12648_gb300 as ipm
    import workloads
    from paper_2005_12648_gb300 import build_ext

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build_ext.build_library()
    ipm.load()
    dist, dt, la, lb, desc = WORKLOADS[args.workload]
    n, w = la + lb, np.dtype(NP_DT[dt]).itemsize
    stream = torch.cuda.current_stream()

    pristine = workloads.make_buffer_torch(torch, dist, NP_DT[dt], la, lb, 0, dev)
    buf = torch.empty_like(pristine)
    G, tile = ipm.ipm_merge_plan(la, lb, dt)
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, dt), dev)

    mb = method_bytes(n, w)

    def step():
        buf.copy_(pristine)
        ipm.ipm_merge_inplace(buf, la, lb, dt, ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ipm.ipm_read_device_status(ws) != 0:
        raise RuntimeError("device status not OK after warm-up")

    sampler = ClockSampler(gpu_uuid(torch)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ipm.ipm_timing_read()  # drop anything recorded before
    ipm.ipm_timing_enable(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for s, e in evs:
        buf.copy_(pristine)
        s.record(stream)
        ipm.ipm_merge_inplace(buf, la, lb, dt, ws)
        e.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ipm.ipm_timing_enable(False)
    phases = ipm.ipm_timing_read().as_dict()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    total_ms = sum(s.elapsed_time(e) for s, e in evs)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = n * world / (ms_per_step * 1e-3) / 1e9
    if ipm.ipm_read_device_status(ws) != 0:
        raise RuntimeError("device status not OK after the timed steps")

    # sanity: the last step's output is sorted (cheap device check; parity is in tests)
    ok_sorted = bool((buf[1:] >= buf[:-1]).all().item()) if dt == "int32" else None

    peak, peak_kind = peaks()
    exch = phases["exchange"]
    exch_launch_ms = exch["ms"] / max(1, exch["launches"])
    launches_per_step = exch["launches"] // args.steps
    # the library's own count of the exchange's algorithmic bytes for this input
    mb["exchange"] = ipm.ipm_read_exchange_bytes(ws)
    mb["total"] = mb["exchange"] + mb["merge"]
    exch_bytes_per_launch = mb["exchange"] / max(1, launches_per_step)
    achieved = exch_bytes_per_launch / (exch_launch_ms * 1e-3) / 1e9 if exch["ms"] else 0.0
    merge_ms = phases["merge"]["ms"] / max(1, phases["merge"]["launches"])
    merge_gbs = mb["merge"] / (merge_ms * 1e-3) / 1e9 if merge_ms else 0.0
    gpu_launches = sum(v["launches"] for v in phases.values())

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, ipm, pristine, la, lb, dt, ws, args.steps, stream)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        v, sample, reps, _ = cpu_oracle_timing(WORKLOADS[args.workload], budget_s=10.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    step_s = ms_per_step * 1e-3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dt,
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "form": "plain",
                   "log2_pairs": G, "tile_capacity": tile,
                   "l2": "inputs larger than L2 (%.1f GiB buffer)" % (n * w / 2**30)
                   if n * w > (129 << 20) else "L2-resident input (no flush)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "exchange_level_kernel (one launch per level)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "traffic": None,
                     "bytes_per_launch": exch_bytes_per_launch,
                     "launch_ms": exch_launch_ms},
        "path": {"method_bytes": mb["total"], "min_bytes": mb["min"],
                 "method_frac": mb["total"] / step_s / 1e9 / peak,
                 "min_frac": mb["min"] / step_s / 1e9 / peak,
                 "merge_kernel_gbs": merge_gbs, "merge_kernel_frac": merge_gbs / peak,
                 "phase_ms_per_step": {k: v["ms"] / args.steps for k, v in phases.items()}},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "sorted_check": ok_sorted,
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)


def run_e2e(torch, ipm, pristine, la, lb, dt, ws, steps, stream):
    """Same merge through the public API with host buffers: H2D of the input from
    pinned memory, the merge, D2H of the result into pinned memory, all timed."""
    host_in = pristine.cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dbuf = torch.empty_like(pristine)
    for _ in range(2):
        dbuf.copy_(host_in, non_blocking=True)
        ipm.ipm_merge_inplace(dbuf, la, lb, dt, ws)
        host_out.copy_(dbuf, non_blocking=True)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for s, e in evs:
        s.record(stream)
        dbuf.copy_(host_in, non_blocking=True)
        ipm.ipm_merge_inplace(dbuf, la, lb, dt, ws)
        host_out.copy_(dbuf, non_blocking=True)
        e.record(stream)
    torch.cuda.synchronize()
    ms = sum(s.elapsed_time(e) for s, e in evs) / steps
    nbytes = pristine.numel() * pristine.element_size()
    return {"value": (la + lb) / (ms * 1e-3) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": ms}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
