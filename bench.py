#!/usr/bin/env python3
"""Benchmark of the GB300 parallel in-place merge (one JSON line on rank 0).

Default workload: one stable in-place merge of int32 keys, L_A = L_B = 2^28, each run
sorted uniform values in [0, 2^31), one contiguous buffer A|B (2 GiB, larger than L2).
A step is one ipm_merge_inplace call (early exit + split + exchange levels + pair
merge).  The merge destroys its input, so before each step the buffer is restored from a
pristine device copy outside the timed interval; each step is timed with CUDA events on
the launching stream and the K step times are summed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c2-int32-uniform|c2-int32-dup16|...|c4-int32-batched|
                              c5-float32-learned] [--no-forms]

The line also carries "forms": the other two forms of the metric measured in the same
run on their own workloads -- "batched" (20,000 int32 segments, log-uniform lengths,
2^28 keys in all, one ipm_merge_batched call per step, against a loop of
ipm_merge_inplace calls) and "learned" (float32 Gaussian-mixture runs of 2^28 each:
the split step with model proposals against the plain split, P = 2^16, and the whole
merge with each).  --workload c4-int32-batched / c5-float32-learned makes that form
the headline instead.

N > 1 (torchrun): the merge does not shard (a single merge needs an all-to-all that
would defeat "in place"), so every rank merges its own replica; value = all ranks' keys
/ the slowest rank's time, scaling "weak".  --impl reference times the CPU oracle (the
plain sequential merge) on a bounded sample of the same workload on host cores.
"""
from __future__ import annotations

import argparse
import json
import math
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
    "c2-int64-uniform": ("uniform", "int64", 1 << 28, 1 << 28,
                         "int64 L_A=L_B=2^28, uniform over the full signed range"),
    "c3-uint32-kv-zipf": ("zipf", "uint32", 1 << 26, 1 << 26,
                          "key-value: uint32 keys Zipf(1.2) over 2^20 ranks, uint32 payload = "
                          "original buffer index, L_A=L_B=2^26; ipm_merge_inplace_kv"),
    "f1-uint64-kv64-uniform": ("uniform", "uint64", 1 << 27, 1 << 27,
                               "key-value: uint64 keys uniform [0,2^64), uint64 payload = "
                               "original buffer index, L_A=L_B=2^27; ipm_merge_inplace_kv"),
    "c1-int32-uniform": ("uniform", "int32", 1 << 20, 1 << 20,
                         "int32 L_A=L_B=2^20, uniform (L2-resident, 8 MiB)"),
    "c2s-int32-uniform": ("uniform", "int32", 1 << 25, 1 << 25,
                          "int32 L_A=L_B=2^25, uniform (reduced c2 for profiling; 256 MiB)"),
    "c4-int32-batched": ("uniform", "int32", 1 << 27, 1 << 27,
                         "batched: 20,000 int32 segments back to back, per-side lengths "
                         "log-uniform on [2^4, 2^e_max] with e_max set so the total is "
                         "<= 2^28 keys, uniform values; one ipm_merge_batched call"),
    "c5-float32-learned": ("gmm", "float32", 1 << 28, 1 << 28,
                           "learned split: float32 keys from an 8-component Gaussian "
                           "mixture, L_A=L_B=2^28, model trained on 4,096 diagonals "
                           "(300 Adam steps); ipm_merge_inplace_learned"),
}
FORM = {"c4-int32-batched": "batched", "c5-float32-learned": "learned"}

# DRAM bytes (read + write) per launch of exchange_level_ws_kernel on a workload, from
# one single-pass ncu capture of that workload (dram__bytes_read.sum +
# dram__bytes_write.sum, mean of 6 launches).  Valid for the kernel as captured; any
# change to it voids the figure (the last capture, 2,104,150,869 B on c2-int32-uniform,
# was of the kernel with 104 KB stages; the stages are 112 KB now, so none is stored).
EXCHANGE_TRAFFIC = {}
# key-value workloads: the payload type per workload (payload = original buffer index)
KV_WORKLOADS = {"c3-uint32-kv-zipf": "uint32", "f1-uint64-kv64-uniform": "uint64"}
NP_DT = {"int32": np.int32, "uint32": np.uint32, "uint64": np.uint64, "float32": np.float32,
         "int64": np.int64}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c2-int32-uniform", choices=sorted(WORKLOADS))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true",
                   help="skip the batched / learned side measurements")
    p.add_argument("--batched-form", type=int, default=0, choices=[0, 1, 2],
                   help="batched workload: launch form of the timed call (0 = default)")
    p.add_argument("--loop-segments", type=int, default=None,
                   help="batched workload: segments in the loop-of-plain-calls baseline "
                        "(default all; 0 skips it)")
    p.add_argument("--no-tune", action="store_true",
                   help="batched workload: skip the autotuner")
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

def host_cpu() -> dict:
    """The host the CPU numbers ran on: its logical CPU count and model name."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001 - lscpu missing: fall back to /proc/cpuinfo
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform

    return {"host_cpus": os.cpu_count(), "cpu_model": model or platform.machine(),
            "arch": platform.machine()}


def spread(times_ms) -> dict:
    """Median and 10th / 90th percentiles of per-step times (ms)."""
    q = np.percentile(np.asarray(times_ms, dtype=np.float64), [10, 50, 90])
    return {"median": float(q[1]), "p10": float(q[0]), "p90": float(q[2]),
            "n": len(times_ms)}


def method_bytes(n: int, w: int) -> dict:
    """Algorithmic bytes of the pair merge (every key read and written once) and of an
    out-of-place merge; the exchange's bytes come from the library after a run."""
    return {"exchange": 0, "merge": 2 * n * w, "total": 2 * n * w, "min": 2 * n * w}


# ------------------------------------------------------------------ reference arm

def cpu_oracle_timing(wl, budget_s: float = 10.0, steps: int | None = None,
                      warmup: int = 0):
    """The oracle's plain sequential merge on a 2^24+2^24-key sample of the workload
    (same generator), single thread; for the batched workload, the oracle merging the
    first 1/16 of the segments one by one.  Returns (GKeys/s, sample description,
    reps, seconds)."""
    import oracle
    import workloads

    if wl is WORKLOADS["c4-int32-batched"]:
        la, lb, _ = workloads.batched_lengths()
        k = la.size // 16
        buf, offs = workloads.batched_buffer(la[:k], lb[:k], seed=0)
        segs = [(int(o), int(x), int(y)) for o, x, y in zip(offs, la[:k], lb[:k])]
        keys = int(buf.size)

        def once():
            for o, x, y in segs:
                oracle.merge(buf[o:o + x], buf[o + x:o + x + y])

        once()
        times = []
        t_end = time.perf_counter() + budget_s
        while True:
            t0 = time.perf_counter()
            once()
            times.append(time.perf_counter() - t0)
            if (steps is not None and len(times) >= steps) or \
                    (steps is None and time.perf_counter() > t_end):
                break
        tot = sum(times)
        sample = (f"oracle two-pointer merge of the first {k} of the {la.size} segments "
                  f"({keys} keys, 1/16 of the segments), one by one, {len(times)} reps, "
                  f"1 thread")
        return keys * len(times) / tot / 1e9, sample, len(times), tot

    dist, dt, la, lb, _ = wl
    vdt = next((KV_WORKLOADS[k] for k, v in WORKLOADS.items()
                if v is wl and k in KV_WORKLOADS), None)
    kv = vdt is not None
    scale = max(1, (la + lb) // (1 << 25))
    sa, sb = max(1, la // scale), max(1, lb // scale)
    a, b = workloads.make_pair(dist, NP_DT[dt], sa, sb, seed=0)
    va = np.arange(sa, dtype=NP_DT[vdt] if kv else np.uint32)
    vb = np.arange(sa, sa + sb, dtype=NP_DT[vdt] if kv else np.uint32)

    def merge_once():
        if kv:
            oracle.merge_kvw(a, va, b, vb)
        else:
            oracle.merge(a, b)

    oracle.merge(a[:1024], b[:1024])
    for _ in range(warmup):
        merge_once()
    times = []
    t_end = time.perf_counter() + budget_s
    while True:
        t0 = time.perf_counter()
        merge_once()
        times.append(time.perf_counter() - t0)
        if steps is not None:
            if len(times) >= steps:
                break
        elif time.perf_counter() > t_end:
            break
    tot = sum(times)
    sample = (f"oracle two-pointer merge{' (key-value)' if kv else ''} on L_A={sa}, "
              f"L_B={sb} keys of the same generator (1/{scale} of the workload), "
              f"{len(times)} reps, 1 thread")
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
                         "sample": sample, **host_cpu()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t0,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def max_over_ranks(torch, value, world, device):
    """The largest of every rank's value (the slowest rank's time); the value itself on
    one rank."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(keys_per_rank, world, ms_per_step):
    """Whole-job GKeys/s of N replicas: every rank's keys over the slowest rank's time."""
    return keys_per_rank * world / (ms_per_step * 1e-3) / 1e9


def e2e_over_ranks(torch, e2e, world, device):
    """The end-to-end figure of N replicas (every rank measured its own): every rank's
    keys over the slowest rank's step time; one rank's figure unchanged."""
    if e2e is None or world <= 1:
        return e2e
    out = dict(e2e)
    out["ms_per_step"] = max_over_ranks(torch, e2e["ms_per_step"], world, device)
    out["value"] = job_throughput(e2e["keys_per_step"], world, out["ms_per_step"])
    return out


def timed_steps(torch, stream, steps, prep, call):
    """CUDA-event time (ms) of `call` per step, with `prep` (the input restore) run
    before each step outside the timed interval."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for s, e in evs:
        prep()
        s.record(stream)
        call()
        e.record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in evs]


def measure_batched(torch, ipm, workloads, dev, stream, steps, warmup, options=None,
                    loop_segments=None, tune=True):
    """The batched form: 20,000 int32 segments (2^28 keys) merged by one
    ipm_merge_batched call per step; also replayed as a captured CUDA graph, compared
    with a loop of ipm_merge_inplace calls over the segments (all of them unless
    loop_segments is given), and, when tune is set, timed again with the option set
    the library's autotuner picks for this table."""
    la, lb, emax = workloads.batched_lengths()
    pristine, offs = workloads.batched_buffer_torch(torch, la, lb, 0, dev)
    n = pristine.numel()
    buf = torch.empty_like(pristine)
    segs = ipm.segment_table(offs.astype(np.int64), la, lb, dev)
    ws = ipm.workspace(ipm.ipm_merge_batched_workspace_bytes(n, la.size, "int32", False,
                                                             options), dev)

    def prep():
        buf.copy_(pristine)

    def call():
        ipm.ipm_merge_batched(buf, None, n, segs, la.size, "int32", ws, options=options)

    for _ in range(max(1, warmup)):
        prep()
        call()
    torch.cuda.synchronize()
    if ipm.ipm_read_device_status(ws) != 0:
        raise RuntimeError("batched: device status not OK")
    ipm.ipm_timing_read()
    ipm.ipm_timing_enable(True)
    times = timed_steps(torch, stream, steps, prep, call)
    ipm.ipm_timing_enable(False)
    ph = ipm.ipm_timing_read().as_dict()["batched"]
    if ipm.ipm_read_device_status(ws) != 0:
        raise RuntimeError("batched: device status not OK")
    merge_b, exch_b = ipm.ipm_read_merge_bytes(ws), ipm.ipm_read_exchange_bytes(ws)
    ms = statistics.median(times)

    # the same call captured in a CUDA graph
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        prep()
        ipm.ipm_merge_batched(buf, None, n, segs, la.size, "int32", ws, options=options,
                              stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        ipm.ipm_merge_batched(buf, None, n, segs, la.size, "int32", ws, options=options,
                              stream=side)
    gtimes = timed_steps(torch, stream, steps, prep, g.replay)
    if ipm.ipm_read_device_status(ws) != 0:
        raise RuntimeError("batched graph: device status not OK")
    ok_sorted = bool(all((buf[o + 1:o + x + y] >= buf[o:o + x + y - 1]).all().item()
                         for o, x, y in zip(offs[:64].tolist(), la[:64].tolist(),
                                            lb[:64].tolist())))

    # the autotuner's pick for this table (timed on `buf` as scratch, no cache file),
    # then timed like the defaults
    autotuned = None
    if tune:
        tws = ipm.workspace(ipm.ipm_merge_batched_tune_workspace_bytes(n, la.size, "int32"), dev)
        t0 = time.perf_counter()
        res = ipm.ipm_merge_batched_tune(pristine, None, n, segs, la.size, "int32", buf, tws,
                                         reps=5, cache_path="")
        tune_s = time.perf_counter() - t0
        best = res["best"]
        twsb = ipm.workspace(ipm.ipm_merge_batched_workspace_bytes(n, la.size, "int32", False,
                                                                   best), dev)

        def tcall():
            ipm.ipm_merge_batched(buf, None, n, segs, la.size, "int32", twsb, options=best)

        for _ in range(max(1, warmup)):
            prep()
            tcall()
        ttimes = timed_steps(torch, stream, steps, prep, tcall)
        if ipm.ipm_read_device_status(twsb) != 0:
            raise RuntimeError("batched (autotuned options): device status not OK")
        tms = statistics.median(ttimes)
        autotuned = {"options": best, "ms_per_step": tms, "value": n / (tms * 1e-3) / 1e9,
                     "step_ms": spread(ttimes), "default_ms_per_step": ms,
                     "gain_over_default": ms / tms, "tuning_s": tune_s,
                     "search": {k: res[k] for k in ("candidates", "best_ms", "default_ms",
                                                    "table", "signature")}}

    # baseline: one ipm_merge_inplace call per segment, on the first segments
    K = la.size if loop_segments is None else min(loop_segments, la.size)
    kkeys = int((la[:K] + lb[:K]).sum())
    loop_ms = None
    if K > 0:
        wsp = ipm.workspace(ipm.ipm_merge_workspace_bytes(int(la[:K].max()),
                                                          int(lb[:K].max()), "int32"), dev)

        def loop():
            for o, x, y in zip(offs[:K].tolist(), la[:K].tolist(), lb[:K].tolist()):
                ipm.ipm_merge_inplace(buf[o:], x, y, "int32", wsp)

        loop_ms = statistics.median(timed_steps(torch, stream, 2, prep, loop))
    peak, _ = peaks()
    min_b = 2 * n * 4
    return {
        "workload": "c4-int32-batched", "segments": int(la.size), "keys": int(n),
        "e_max": round(float(emax), 4), "max_segment": int((la + lb).max()),
        "options": options or {"tile": 0, "order": 0, "ctas_per_sm": 0, "form": 0},
        "ms_per_step": ms, "value": n / (ms * 1e-3) / 1e9, "unit": UNIT,
        "step_ms": spread(times), "autotuned": autotuned,
        "graph_ms_per_step": statistics.median(gtimes),
        "graph_value": n / (statistics.median(gtimes) * 1e-3) / 1e9,
        "launches_per_step": ph["launches"] // max(1, steps),
        "merge_bytes": merge_b, "exchange_bytes": exch_b, "min_bytes": min_b,
        "method_frac": (merge_b + exch_b) / (ms * 1e-3) / 1e9 / peak,
        "min_frac": min_b / (ms * 1e-3) / 1e9 / peak,
        "loop_baseline": None if loop_ms is None else {
            "segments": K, "keys": kkeys, "ms": loop_ms,
            "value": kkeys / (loop_ms * 1e-3) / 1e9,
            "calls": K, "note": "one ipm_merge_inplace call per segment"},
        "speedup_vs_loop": None if loop_ms is None else
        (n / (ms * 1e-3)) / (kkeys / (loop_ms * 1e-3)),
        "sorted_check": ok_sorted, "buffer": buf, "pristine": pristine,
    }


def measure_learned(torch, ipm, workloads, dev, stream, steps, warmup, P=1 << 16,
                    nsamples=4096, train_steps=300):
    """The learned-split form on float32 Gaussian-mixture runs of 2^28 each: the model
    is trained once (timed), then the split step with proposals is timed against the
    plain split at P diagonals, and the whole merge with each split step."""
    la = lb = 1 << 28
    n = la + lb
    pristine = workloads.make_buffer_torch(torch, "gmm", np.float32, la, lb, 0, dev)
    buf = torch.empty_like(pristine)
    diags = torch.from_numpy(workloads.split_training_diagonals(n, nsamples, 0)
                             .view(np.int64)).to(dev)
    model = ipm.split_model_to_device(ipm.split_model_initial_params(), dev)
    tws = ipm.workspace(ipm.ipm_split_model_train_workspace_bytes(nsamples), dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    ipm.ipm_split_model_train(pristine, la, lb, "float32", diags, nsamples, model, tws,
                              steps=train_steps, lr=1e-2)
    t1.record(stream)
    torch.cuda.synchronize()
    train_ms = t0.elapsed_time(t1)
    _, loss, _ = ipm.split_model_from_device(model)

    out = torch.empty(P + 1, dtype=torch.int64, device=dev)
    ref = torch.empty(P + 1, dtype=torch.int64, device=dev)
    split = {}
    for name, m in (("plain", None), ("learned", model)):
        st = torch.zeros(5, dtype=torch.int64, device=dev)
        ipm.ipm_merge_splits_learned(pristine, la, lb, "float32", P, m, out, st)
        torch.cuda.synchronize()
        stats = st.cpu().numpy()
        if name == "plain":
            call = (lambda: ipm.ipm_merge_splits(pristine, la, lb, "float32", P, ref))
        else:
            call = (lambda: ipm.ipm_merge_splits_learned(pristine, la, lb, "float32", P,
                                                         model, out))
        for _ in range(3):
            call()
        t = statistics.median(timed_steps(torch, stream, max(5, steps), lambda: None, call))
        split[name] = {"ms": t, "rounds_per_split": float(stats[1] / stats[0]),
                       "probes_per_split": float(stats[2] / stats[0]),
                       "mean_abs_err": float(stats[3] / stats[0]),
                       "max_abs_err": int(stats[4])}
    torch.cuda.synchronize()
    same = bool(torch.equal(out, ref))

    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, "float32"), dev)
    calls = {"plain": lambda: ipm.ipm_merge_inplace(buf, la, lb, "float32", ws),
             "learned": lambda: ipm.ipm_merge_inplace_learned(buf, la, lb, "float32", model,
                                                              ws)}
    for _ in range(max(1, warmup)):
        for call in calls.values():
            buf.copy_(pristine)
            call()
    # the two forms alternate step by step on the same buffer, so a drift of the clock
    # or of the memory system affects both alike
    times = {"plain": [], "learned": []}
    split_ms = {"plain": 0.0, "learned": 0.0}
    launches = {"plain": 0, "learned": 0}
    for _ in range(steps):
        for name, call in calls.items():
            ipm.ipm_timing_read()
            ipm.ipm_timing_enable(True)
            times[name] += timed_steps(torch, stream, 1, lambda: buf.copy_(pristine), call)
            ipm.ipm_timing_enable(False)
            ph = ipm.ipm_timing_read().as_dict()
            split_ms[name] += ph["learned_split" if name == "learned" else "split"]["ms"]
            launches[name] += sum(v["launches"] for v in ph.values())
            if ipm.ipm_read_device_status(ws) != 0:
                raise RuntimeError(f"learned form ({name}): device status not OK")
    merges = {}
    for name in calls:
        sp = spread(times[name])
        merges[name] = {"ms_per_step": sp["median"], "value": n / (sp["median"] * 1e-3) / 1e9,
                        "step_ms": sp, "split_phase_ms": split_ms[name] / steps,
                        "launches_per_step": launches[name] // steps}
    pl, le = merges["plain"]["step_ms"], merges["learned"]["step_ms"]
    gain = {"median_ratio": pl["median"] / le["median"],
            "ranges_overlap": not (le["p90"] < pl["p10"] or pl["p90"] < le["p10"]),
            "split_phase_saved_ms": merges["plain"]["split_phase_ms"] -
            merges["learned"]["split_phase_ms"]}
    ok_sorted = bool((buf[1:] >= buf[:-1]).all().item())
    return {
        "workload": "c5-float32-learned", "keys": n, "P": P,
        "model": {"hidden": 32, "params": 97, "dtype": "fp32", "train_samples": nsamples,
                  "train_steps": train_steps, "train_ms": train_ms, "train_loss": loss},
        "split": split, "split_speedup": split["plain"]["ms"] / split["learned"]["ms"],
        "splits_identical": same, "merge": merges, "end_to_end_gain": gain,
        "value": merges["learned"]["value"], "ms_per_step": merges["learned"]["ms_per_step"],
        "unit": UNIT, "sorted_check": ok_sorted, "buffer": buf, "pristine": pristine,
        "model_tensor": model,
    }


def measure_rotations(torch, ipm, dev, stream, steps=5, warmup=3):
    """The partition exchange [X|Y] -> [Y|X] of 2^29 uint32 elements (2 GiB, larger
    than L2) by linear shifting (ipm_rotate, the merge's exchange engine) and by
    circular shifting (ipm_rotate_cs), for split points whose cycle counts
    gcd(|X|, |Y|) span the coalesced and the scattered regime; both results are
    compared with each other and with the definition (a roll)."""
    peak, _ = peaks()
    n = 1 << 29
    half = n // 2
    pristine = torch.randint(0, 1 << 31, (n,), dtype=torch.int64, device=dev).to(torch.int32)
    buf = torch.empty_like(pristine)
    out = []
    for lx in (half, half + 64, half + 1):
        ly = n - lx
        res = {"len_x": lx, "len_y": ly, "cycles": math.gcd(lx, ly)}
        kept = {}
        for name, wsq, fn in (("ls", ipm.ipm_rotate_workspace_bytes, ipm.ipm_rotate),
                              ("cs", ipm.ipm_rotate_cs_workspace_bytes, ipm.ipm_rotate_cs)):
            ws = ipm.workspace(wsq(lx, ly, 4), dev)

            def prep():
                buf.copy_(pristine)

            def call():
                fn(buf, lx, ly, 4, ws)

            for _ in range(warmup):
                prep()
                call()
            torch.cuda.synchronize()
            kept[name] = buf.clone()
            ms = float(np.median(timed_steps(torch, stream, steps, prep, call)))
            gbs = 2.0 * n * 4 / (ms * 1e-3) / 1e9
            res[name] = {"ms": ms, "gbs": gbs, "frac": gbs / peak}
            del ws
        want = torch.roll(pristine, -lx)
        res["identical"] = bool(torch.equal(kept["ls"], want) and torch.equal(kept["cs"], want))
        res["cs_over_ls_time"] = res["cs"]["ms"] / res["ls"]["ms"]
        del kept, want
        out.append(res)
    return {"workload": "exchange of 2^29 uint32 elements (2 GiB), split points with "
                        "2^28, 64 and 1 cycles", "bytes_per_call": 2 * n * 4,
            "peak_gbs": peak, "shapes": out}


def _largest_pairs(ia, jb):
    """Largest pair of a division: over the pairs that need a merge (both sides
    non-empty) and over all pairs."""
    na = np.diff(ia.astype(np.int64))
    nb = np.diff(jb.astype(np.int64))
    c = na + nb
    need = (na > 0) & (nb > 0)
    return (int(c[need].max()) if need.any() else 0), int(c.max())


def measure_division(torch, ipm, workloads, dev, stream, steps=10, warmup=3):
    """The balance comparison of Sec. 4 (E1): the division of Alg. 3 by FindMedian
    against the optimal (exact half-diagonal) split, (Max_FM - Max_opt) / Max_opt of
    the largest pair that needs a merge, on the paper's random-walk workload at its
    largest size (2^22 int32 keys) split at 1/4, 1/2, 3/4, for T = 2..16; and at the
    merge's own scale (2^28 + 2^28 uniform int32, T = 2^15), with the time of the
    FindMedian division against the exact splits the merge uses."""
    table = []
    n = 1 << 22
    for frac in (0.25, 0.5, 0.75):
        la = int(n * frac)
        buf = workloads.make_buffer_torch(torch, "paper", np.int32, la, n - la, 4, dev)
        row = {"split_at": frac, "T": [], "rel_diff": [], "rel_diff_all_pairs": []}
        for depth in (1, 2, 3, 4):
            fm = _largest_pairs(*[t.cpu().numpy() for t in ipm.division_splits(
                buf, la, n - la, "int32", depth, "findmedian")])
            ex = _largest_pairs(*[t.cpu().numpy() for t in ipm.division_splits(
                buf, la, n - la, "int32", depth, "exact")])
            row["T"].append(1 << depth)
            row["rel_diff"].append((fm[0] - ex[0]) / ex[0])
            row["rel_diff_all_pairs"].append((fm[1] - ex[1]) / ex[1])
        table.append(row)
        del buf
    la = lb = 1 << 28
    buf = workloads.make_buffer_torch(torch, "uniform", np.int32, la, lb, 0, dev)
    depth = 15
    fm = _largest_pairs(*[t.cpu().numpy() for t in ipm.division_splits(
        buf, la, lb, "int32", depth, "findmedian")])
    ex = _largest_pairs(*[t.cpu().numpy() for t in ipm.division_splits(
        buf, la, lb, "int32", depth, "exact")])
    ia = torch.empty((1 << depth) + 1, dtype=torch.int64, device=dev)
    jb = torch.empty_like(ia)
    split = torch.empty_like(ia)
    times = {}
    for name, call in (
            ("findmedian_division", lambda: ipm.ipm_division_splits(
                buf, la, lb, "int32", depth, "findmedian", ia, jb)),
            ("exact_division", lambda: ipm.ipm_division_splits(
                buf, la, lb, "int32", depth, "exact", ia, jb)),
            ("merge_splits", lambda: ipm.ipm_merge_splits(buf, la, lb, "int32", 1 << depth,
                                                          split))):
        for _ in range(warmup):
            call()
        times[name] = float(np.median(timed_steps(torch, stream, steps, lambda: None, call)))
    return {"workload": "paper random walk x[i] = x[i-1] + floor(5 U), 2^22 int32 keys; "
                        "uniform int32 2^28 + 2^28 at T = 2^15",
            "metric": "(Max_FindMedian - Max_optimal) / Max_optimal, largest pair that "
                      "needs a merge", "paper_workload_2p22": table,
            "uniform_2p29": {"T": 1 << depth, "max_pair_findmedian": fm[0],
                             "max_pair_exact": ex[0], "rel_diff": (fm[0] - ex[0]) / ex[0],
                             "ms": times}}


def measure_permutation(torch, ipm, workloads, dev, stream, steps=5, warmup=3):
    """The division stage by one permutation (sOptMov, Alg. 2) against the level-by-level
    exchange (sRecPar, Alg. 3) on the headline buffer (uniform int32 2^28 + 2^28) with
    the same exact split table: each alone, and each inside a whole merge (splits,
    division, pair merge).  The two layouts are compared with each other."""
    peak, _ = peaks()
    la = lb = 1 << 28
    n = la + lb
    name = "int32"
    pristine = workloads.make_buffer_torch(torch, "uniform", np.int32, la, lb, 0, dev)
    buf = torch.empty_like(pristine)
    G = ipm.ipm_merge_plan(la, lb, name)[0]
    split = torch.empty((1 << G) + 1, dtype=torch.int64, device=dev)
    ipm.ipm_merge_splits(pristine, la, lb, name, 1 << G, split)
    ws_perm = ipm.workspace(ipm.ipm_rearrange_permute_workspace_bytes(la, lb, name), dev)
    ws_lvl = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, name, False, G), dev)
    calls = {
        "permute": lambda: ipm.ipm_rearrange_permute(buf, None, la, lb, name, split, G,
                                                     ws_perm),
        "levels": lambda: ipm.ipm_merge_rearrange(buf, None, la, lb, name, split, G, ws_lvl),
        "merge_via_permute": lambda: (ipm.ipm_merge_splits(buf, la, lb, name, 1 << G, split),
                                      ipm.ipm_rearrange_permute(buf, None, la, lb, name, split,
                                                                G, ws_perm),
                                      ipm.ipm_merge_pairs(buf, None, la, lb, name, split, G)),
        "merge_default": lambda: ipm.ipm_merge_inplace(buf, la, lb, name, ws_lvl),
    }

    def prep():
        buf.copy_(pristine)

    res, kept = {}, {}
    for key, call in calls.items():
        for _ in range(warmup):
            prep()
            call()
        torch.cuda.synchronize()
        kept[key] = buf.clone() if key in ("permute", "levels") else None
        if key.startswith("merge"):
            kept[key] = bool(torch.all(buf[1:] >= buf[:-1]).item())
        ms = float(np.median(timed_steps(torch, stream, steps, prep, call)))
        res[key] = {"ms": ms}
        if key in ("permute", "levels"):
            gbs = 2.0 * n * 4 / (ms * 1e-3) / 1e9
            res[key].update({"gbs_one_pass": gbs, "frac_one_pass": gbs / peak})
        else:
            res[key]["gkeys_s"] = n / (ms * 1e-3) / 1e9
    same = bool(torch.equal(kept["permute"], kept["levels"]))
    del kept["permute"], kept["levels"], buf, pristine, ws_perm, ws_lvl
    return {"workload": "uniform int32 2^28 + 2^28, exact splits, P = 2^%d" % G,
            "bytes_one_pass": 2 * n * 4, "peak_gbs": peak, "ms": res,
            "layouts_identical": same, "merges_sorted": [kept["merge_via_permute"],
                                                         kept["merge_default"]],
            "permute_over_levels_time": res["permute"]["ms"] / res["levels"]["ms"]}


def _public(d):
    return {k: v for k, v in d.items() if k not in ("buffer", "pristine", "model_tensor")}


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
    stream = torch.cuda.current_stream()
    form = FORM.get(args.workload, "plain")
    if form == "plain":
        line = run_plain(args, rank, world, torch, ipm, workloads, dev, stream)
    else:
        line = run_form(args, rank, world, torch, ipm, workloads, dev, stream, form)
    if line is None:
        return
    if not args.no_forms and world == 1:
        torch.cuda.empty_cache()
        forms = {}
        if form != "batched":
            forms["batched"] = _public(measure_batched(torch, ipm, workloads, dev, stream,
                                                       steps=10, warmup=2))
            torch.cuda.empty_cache()
        if form != "learned":
            forms["learned"] = _public(measure_learned(torch, ipm, workloads, dev, stream,
                                                       steps=50, warmup=2))
            torch.cuda.empty_cache()
        forms["rotate"] = measure_rotations(torch, ipm, dev, stream)
        torch.cuda.empty_cache()
        forms["division"] = measure_division(torch, ipm, workloads, dev, stream)
        torch.cuda.empty_cache()
        forms["permutation"] = measure_permutation(torch, ipm, workloads, dev, stream)
        torch.cuda.empty_cache()
        line["forms"] = forms
    print(json.dumps(line), flush=True)


def run_form(args, rank, world, torch, ipm, workloads, dev, stream, form):
    """Headline line of the batched or learned form (replicas when N > 1)."""
    sampler = ClockSampler(gpu_uuid(torch)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    if form == "batched":
        m = measure_batched(torch, ipm, workloads, dev, stream, args.steps, args.warmup,
                            options={"form": args.batched_form} if args.batched_form else None,
                            loop_segments=args.loop_segments, tune=not args.no_tune)
    else:
        m = measure_learned(torch, ipm, workloads, dev, stream, args.steps, args.warmup)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(torch, m["ms_per_step"], world, dev)
    e2e = None
    if not args.no_e2e and form == "learned":
        e2e = run_e2e_learned(torch, ipm, m, args.steps, stream, m["model_tensor"])
    elif not args.no_e2e:
        e2e = run_e2e_batched(torch, ipm, workloads, m, args.steps, stream, dev)
    e2e = e2e_over_ranks(torch, e2e, world, dev)
    if rank != 0:
        return None
    dist, dt, la, lb, desc = WORKLOADS[args.workload]
    n = m["keys"]
    peak, peak_kind = peaks()
    if form == "batched":
        achieved = (m["merge_bytes"] + m["exchange_bytes"]) / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "batched call (levels + merge kernels)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": f"{peak_kind} hbm_gbs", "traffic": None,
                "bytes_per_launch": m["merge_bytes"] + m["exchange_bytes"], "launch_ms": ms}
        launches = m["launches_per_step"] * args.steps
    else:
        exch_note = "exchange_level_ws_kernel (one launch per level), as in the plain form"
        roof = {"bound": "hbm", "kernel": exch_note, "achieved": None, "peak": peak,
                "unit": "GB/s", "frac": None, "peak_kind": f"{peak_kind} hbm_gbs",
                "traffic": None}
        launches = m["merge"]["learned"]["launches_per_step"] * args.steps
    cpu = None
    if not args.no_cpu_baseline:
        v, sample, reps, _ = cpu_oracle_timing(WORKLOADS[args.workload], budget_s=10.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               **host_cpu()}

    return {
        "metric": METRIC, "value": job_throughput(n, world, ms), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dt,
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "form": form,
                   "l2": "inputs larger than L2 (%.1f GiB buffer)" % (n * 4 / 2**30),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof, "form_detail": _public(m), "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks, "sorted_check": m["sorted_check"],
    }


def run_e2e_batched(torch, ipm, workloads, m, steps, stream, dev):
    """The batched call with host buffers: H2D of the keys, the merge, D2H, timed."""
    pristine = m["pristine"]
    la, lb, _ = workloads.batched_lengths()
    offs = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.int64)
    segs = ipm.segment_table(offs, la, lb, dev)
    n = pristine.numel()
    ws = ipm.workspace(ipm.ipm_merge_batched_workspace_bytes(n, la.size, "int32"), dev)
    return run_e2e(torch, [pristine], steps,
                   lambda d, k, st: ipm.ipm_merge_batched(d[0], None, n, segs, la.size, "int32",
                                                          ws, stream=st))


def run_e2e_learned(torch, ipm, m, steps, stream, model):
    pristine = m["pristine"]
    la = lb = pristine.numel() // 2
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, "float32"), pristine.device)
    return run_e2e(torch, [pristine], steps,
                   lambda d, k, st: ipm.ipm_merge_inplace_learned(d[0], la, lb, "float32", model,
                                                                  ws, stream=st))


def run_plain(args, rank, world, torch, ipm, workloads, dev, stream):
    dist, dt, la, lb, desc = WORKLOADS[args.workload]
    kv = args.workload in KV_WORKLOADS
    vdt = KV_WORKLOADS.get(args.workload)
    vbytes = 8 if vdt == "uint64" else (4 if kv else 0)
    n, w = la + lb, np.dtype(NP_DT[dt]).itemsize + vbytes

    pristine = workloads.make_buffer_torch(torch, dist, NP_DT[dt], la, lb, 0, dev)
    buf = torch.empty_like(pristine)
    # key-value: payload = the key's original buffer index
    vpristine = None
    if kv:
        vpristine = torch.arange(n, dtype=torch.int64, device=dev)
        if vbytes == 4:
            vpristine = vpristine.to(torch.int32)
    vbuf = torch.empty_like(vpristine) if kv else None
    G, tile = ipm.ipm_merge_plan(la, lb, dt, with_values=vbytes)
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, dt, with_values=vbytes), dev)

    mb = method_bytes(n, w)

    def merge(kb, vb=None, w=None, stream=None):
        w = ws if w is None else w
        if kv:
            ipm.ipm_merge_inplace_kv(kb, vb, la, lb, dt, w, val_dtype=vdt, stream=stream)
        else:
            ipm.ipm_merge_inplace(kb, la, lb, dt, w, stream=stream)

    def restore():
        buf.copy_(pristine)
        if kv:
            vbuf.copy_(vpristine)

    def step():
        restore()
        merge(buf, vbuf)

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
        restore()
        s.record(stream)
        merge(buf, vbuf)
        e.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ipm.ipm_timing_enable(False)
    phases = ipm.ipm_timing_read().as_dict()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    step_times = [s.elapsed_time(e) for s, e in evs]
    total_ms = max_over_ranks(torch, sum(step_times), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(n, world, ms_per_step)
    if ipm.ipm_read_device_status(ws) != 0:
        raise RuntimeError("device status not OK after the timed steps")

    # sanity: the last step's output is sorted (cheap device check; parity is in tests);
    # key-value: equal keys keep their payloads (original indices) ascending
    ok_sorted = None
    if dt in ("int32", "int64") and not kv:
        ok_sorted = bool((buf[1:] >= buf[:-1]).all().item())
    elif kv and dt in ("uint32", "uint64"):
        # unsigned order as signed order (uint64: flip the top bit; uint32: widen)
        k64 = (buf.to(torch.int64) & 0xFFFFFFFF) if dt == "uint32" else (buf ^ (-(1 << 63)))
        ok_sorted = bool(((k64[1:] > k64[:-1]) |
                          ((k64[1:] == k64[:-1]) & (vbuf[1:] > vbuf[:-1]))).all().item())
        del k64

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
        e2e = run_e2e(torch, [pristine, vpristine] if kv else [pristine], args.steps,
                      lambda d, k, st: merge(d[0], d[1] if kv else None, ws, st))
        e2e = e2e_over_ranks(torch, e2e, world, dev)
    del buf, pristine, vbuf, vpristine

    if rank != 0:
        return None
    cpu = None
    if not args.no_cpu_baseline:
        v, sample, reps, _ = cpu_oracle_timing(WORKLOADS[args.workload], budget_s=10.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               **host_cpu()}
    step_s = ms_per_step * 1e-3
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "step_ms": spread(step_times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{dt} key + {vdt} payload" if kv else dt,
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc,
                   "form": "key-value" if kv else "plain",
                   "log2_pairs": G, "tile_capacity": tile,
                   "fused": dict(zip(("engine", "levels"),
                                     ipm.ipm_merge_fused_plan(la, lb, dt, vbytes))),
                   "l2": "inputs larger than L2 (%.1f GiB buffer)" % (n * w / 2**30)
                   if n * w > (129 << 20) else "L2-resident input (no flush)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm",
                     "kernel": "exchange_level_ws_kernel (one launch per exchange level)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "traffic": EXCHANGE_TRAFFIC.get(args.workload),
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


def run_e2e(torch, pristines, steps, merge, slots=3):
    """The merge through the public API with host buffers, as a caller merging a stream
    of inputs runs it: every step copies its input (keys, and payloads for key-value)
    from pinned host memory, merges it and copies the result back to pinned host memory.
    Three streams carry the copies in, the merges and the copies back; `slots` sets of
    device buffers rotate between them (a buffer's next copy in waits for its last copy
    back), so one step's copy in, another's merge and a third's copy back run at once
    and the link carries both directions together.  The merges run one after another on
    their stream, so one workspace serves them (merge(device buffers, slot, stream)); the
    copies back run in order on theirs, so one set of pinned output buffers serves them.
    Timed from before the first copy in to after the last copy back."""
    host_in = [p.cpu().pin_memory() for p in pristines]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    dbuf = [[torch.empty_like(p) for p in pristines] for _ in range(slots)]
    s_in, s_merge, s_out = (torch.cuda.Stream() for _ in range(3))
    ev_in = [torch.cuda.Event() for _ in range(slots)]
    ev_merged = [torch.cuda.Event() for _ in range(slots)]
    ev_out = [torch.cuda.Event() for _ in range(slots)]
    used = [False] * slots

    def step(k):
        q = k % slots
        if used[q]:
            s_in.wait_event(ev_out[q])  # the buffers' previous result has been read back
        with torch.cuda.stream(s_in):
            for d, h in zip(dbuf[q], host_in):
                d.copy_(h, non_blocking=True)
            ev_in[q].record(s_in)
        s_merge.wait_event(ev_in[q])
        merge(dbuf[q], q, s_merge)
        ev_merged[q].record(s_merge)
        s_out.wait_event(ev_merged[q])
        with torch.cuda.stream(s_out):
            for h, d in zip(host_out, dbuf[q]):
                h.copy_(d, non_blocking=True)
            ev_out[q].record(s_out)
        used[q] = True

    for k in range(slots):
        step(k)
    torch.cuda.synchronize()
    start, end = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    start.record(s_in)
    s_merge.wait_event(start)
    s_out.wait_event(start)
    for k in range(steps):
        step(k)
    end.record(s_out)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end) / steps
    nbytes = sum(p.numel() * p.element_size() for p in pristines)
    return {"value": pristines[0].numel() / (ms * 1e-3) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": ms,
            "keys_per_step": pristines[0].numel(),
            "pipelined": f"{slots} buffer sets over three streams (copy in, merge, copy back)"}


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
