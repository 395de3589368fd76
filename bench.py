#!/usr/bin/env python
"""Benchmark of the STREAM hot path on B300 (Heller et al., Section 5, Listing 4).

One step = one STREAM pass (Copy c=a, Scale b=c*q, Add c=a+b, Triad a=b+c*q; q=3) over three
device-resident FP64 arrays of n = 2^27 elements (1 GiB each, far beyond the 126 MB L2, so no
L2 flush is needed between steps), seeded uniform in [-1, 1).  ``value`` is the STREAM byte
count of the pass (copy/scale 2*n*8 B, add/triad 3*n*8 B) over the device time, summed over
ranks (weak scaling: every rank runs its own arrays; no collective on the data path).

Also reported on the same JSON line: per-kernel GB/s (FP64 and FP32), the roofline of the
dominant kernel (Triad) against the measured HBM copy bandwidth, the end-to-end figure through
the C ABI from pinned host buffers, the CPU oracle on a bounded sample, SM clocks sampled during
the timed region, and (sections "batched" and "served") the persistent batched launcher vs one
launch per instance and the continuous-batching server vs a per-call FIFO.

``--impl reference`` times the CPU oracle (serial C, one core) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "copy/triad HBM GB/s and % of B300 peak; batched vs per-call p50/p99 latency"
FALLBACK_HBM_GBS = 6400.0
NOMINAL_HBM_GBS = 8000.0
Q = 3.0

# dram__bytes_read.sum + dram__bytes_write.sum of one Triad launch (FP64, n = 2^27) from an ncu
# capture, with the sha256 of the kernel source it was taken on; reported as null when the
# source has changed since.
NCU_TRAFFIC = {"kernel": "k_stream_vec<TRIAD,double>", "n": 1 << 27, "bytes": None,
               "source_sha256": None}


def _rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _kernel_source_sha():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2206_06302_b300", "csrc", "sx_kernels.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------------------------

def cpu_oracle_gbs(n: int, seconds: float):
    """The serial oracle's STREAM pass on a sample of n FP64 elements, repeated for ~seconds."""
    import oracle
    import stream_inputs as si
    a, b, c = si.stream_arrays(n, np.float64)
    oracle.stream(a, b, c, Q, 1)  # warm (page in)
    passes, t0 = 0, time.perf_counter()
    while True:
        oracle.stream(a, b, c, Q, 1)
        passes += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return 10.0 * n * 8 * passes / el / 1e9, passes, el


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    import oracle
    import stream_inputs as si
    n = args.ref_n
    a, b, c = si.stream_arrays(n, np.float64)
    for _ in range(args.warmup):
        oracle.stream(a, b, c, Q, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.stream(a, b, c, Q, 1)
    el = time.perf_counter() - t0
    gbs = 10.0 * n * 8 * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic: seeded SplitMix64 uniform [-1,1)",
        "config": {"workload": f"STREAM FP64 pass (copy,scale,add,triad), q=3, bounded sample "
                               f"n={n} per array of the n=2^27 workload", "n": n},
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"n={n} FP64 per array, {args.steps} passes"},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------
# GPU legs
# ----------------------------------------------------------------------------------------------

def stream_kernels(sx, torch, t, stream, e, dtype_code, n, steps, warmup, seed_instance):
    """Per-kernel device times of `steps` STREAM passes; returns dict and total elapsed ms."""
    import stream_inputs as si
    es = 8 if dtype_code == sx.SX_F64 else 4
    arrs = [sx.sx_alloc(t, dtype_code, n) for _ in range(3)]
    for k, arr in enumerate(arrs):
        sx.sx_seed_uniform(arr, si.array_seed(si.BASE_SEED, k, seed_instance), -1.0, 1.0)
    a, b, c = arrs
    seq = [("copy", sx.SX_OP_COPY, a, None, c), ("scale", sx.SX_OP_SCALE, c, None, b),
           ("add", sx.SX_OP_ADD, a, b, c), ("triad", sx.SX_OP_TRIAD, b, c, a)]

    def one_pass(evs=None):
        if evs is not None:
            evs[0].record(stream)
        for k, (_, op, x, y, o) in enumerate(seq):
            sx.sx_execute_async(e, op, x, y, o, Q, future=False)
            if evs is not None:
                evs[k + 1].record(stream)

    for _ in range(warmup):
        one_pass()
    torch.cuda.synchronize()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    return arrs, seq, one_pass, events, es


def run_ours(args):
    import torch
    import paper_2206_06302_b300 as sx

    rank, world, local = _rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(local)
    t = sx.target_on_torch_stream(local, stream)
    info = sx.sx_target_info_get(t)
    n = args.n
    tuned = {}
    if args.tune:
        if args.tune_cache and os.path.exists(args.tune_cache):
            sx.sx_tune_load(args.tune_cache)
        for dcode in (sx.SX_F64, sx.SX_F32):
            for name, op in (("copy", sx.SX_OP_COPY), ("scale", sx.SX_OP_SCALE),
                             ("add", sx.SX_OP_ADD), ("triad", sx.SX_OP_TRIAD)):
                if sx.sx_tune_lookup(t, op, dcode, n) is None:
                    sx.sx_tune(t, op, dcode, n)
        if args.tune_cache:
            sx.sx_tune_save(args.tune_cache)
    e = sx.sx_executor_create(t, sx.SX_PAR_TASK)
    for dcode, dname in ((sx.SX_F64, "f64"), (sx.SX_F32, "f32")):
        tuned[dname] = {name: sx.sx_executor_resolve(e, op, dcode, n) for name, op in
                        (("copy", 0), ("scale", 1), ("add", 2), ("triad", 3))}

    peak, peak_kind = _measured_peaks()
    out = {}

    # ---- the timed region: FP64 STREAM passes ------------------------------------------------
    arrs, seq, one_pass, events, es = stream_kernels(
        sx, torch, t, stream, e, sx.SX_F64, n, args.steps, args.warmup, rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for s in range(args.steps):
            one_pass(events[s])
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sx.sx_target_synchronize(t)  # surfaces any device-side error word
    per = {name: 0.0 for name, *_ in seq}
    for s in range(args.steps):
        for k, (name, *_r) in enumerate(seq):
            per[name] += events[s][k].elapsed_time(events[s][k + 1])
    total_ms = events[0][0].elapsed_time(events[-1][-1])
    if dist:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    step_bytes = 10.0 * n * es
    value = world * step_bytes * args.steps / (total_ms * 1e-3) / 1e9
    bytes_per = {"copy": 2, "scale": 2, "add": 3, "triad": 3}
    kernels = {}
    for name in per:
        ms = per[name] / args.steps
        gbs = bytes_per[name] * n * es / (ms * 1e-3) / 1e9
        kernels[name] = {"ms": round(ms, 5), "GB/s": round(gbs, 1),
                         "frac_measured": round(gbs / peak, 4),
                         "frac_nominal_8TBs": round(gbs / NOMINAL_HBM_GBS, 4)}
    clk = clocks.summary()

    # ---- FP32 per-kernel figures (same shape, fewer steps) -----------------------------------
    kernels_f32 = None
    if not args.quick:
        for arr in arrs:
            sx.sx_free(arr)
        steps32 = max(3, min(args.steps, 200))
        arrs, seq, one_pass, ev32, es32 = stream_kernels(
            sx, torch, t, stream, e, sx.SX_F32, n, steps32, args.warmup, rank)
        for s in range(steps32):
            one_pass(ev32[s])
        torch.cuda.synchronize()
        kernels_f32 = {}
        for k, (name, *_r) in enumerate(seq):
            ms = sum(ev32[s][k].elapsed_time(ev32[s][k + 1]) for s in range(steps32)) / steps32
            gbs = bytes_per[name] * n * es32 / (ms * 1e-3) / 1e9
            kernels_f32[name] = {"ms": round(ms, 5), "GB/s": round(gbs, 1),
                                 "frac_measured": round(gbs / peak, 4)}
    for arr in arrs:
        sx.sx_free(arr)

    # ---- end to end through the C ABI from pinned host buffers --------------------------------
    e2e = None
    if not args.quick and args.e2e_steps > 0:
        import stream_inputs as si
        host = []
        for k in range(3):
            h = torch.empty(n, dtype=torch.float64, pin_memory=True)
            h.numpy()[:] = si.uniform(si.array_seed(si.BASE_SEED, k, rank), n, np.float64) if k == 0 \
                else 0.0
            host.append(h)
        dev = [sx.sx_alloc(t, sx.SX_F64, n) for _ in range(3)]
        esync = sx.sx_executor_create(t, sx.SX_PAR)
        sx.sx_stream_host(esync, *(h.data_ptr() for h in host), *dev, Q, 1)  # warm
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sx.sx_stream_host(esync, *(h.data_ptr() for h in host), *dev, Q, 1)
        el = time.perf_counter() - t0
        if dist:
            tt = torch.tensor([el], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        e2e = {"value": round(world * step_bytes * args.e2e_steps / el / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": 3 * n * 8, "d2h_bytes_per_step": 3 * n * 8,
               "steps": args.e2e_steps,
               "what": "sx_stream_host: h2d a,b,c + one pass (4 launches) + d2h a,b,c, host clock"}
        for d in dev:
            sx.sx_free(d)
        sx.sx_executor_destroy(esync)
        del host

    # ---- sections beyond the plain pass --------------------------------------------------------
    extra = {}
    if not args.quick and "batched" in args.sections:
        from bench_sections import batched_section
        extra["batched"] = batched_section(sx, torch, t, stream, args)
    if not args.quick and "served" in args.sections:
        from bench_sections import served_section
        extra["served"] = served_section(sx, torch, t, stream, args)

    # ---- CPU oracle on a bounded sample (rank 0, N=1 only) ------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        gbs, passes, el = cpu_oracle_gbs(args.cpu_n, args.cpu_seconds)
        cpu = {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"STREAM FP64 pass on n={args.cpu_n} per array, {passes} passes "
                         f"in {el:.1f} s (serial C, -O2 -ffp-contract=off)"}

    triad_ms = per["triad"] / args.steps
    achieved = 3 * n * es / (triad_ms * 1e-3) / 1e9
    traffic = None
    if NCU_TRAFFIC["bytes"] and NCU_TRAFFIC["source_sha256"] == _kernel_source_sha() \
            and NCU_TRAFFIC["n"] == n:
        traffic = NCU_TRAFFIC["bytes"]
    roofline = {"bound": "hbm", "kernel": "triad f64", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "frac_nominal_8TBs": round(achieved / NOMINAL_HBM_GBS, 4),
                "algorithmic_bytes_per_launch": 3 * n * es, "traffic": traffic}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded SplitMix64 uniform [-1,1), constructed on the device",
            "config": {"workload": "STREAM FP64 n=2^27 per array (1 GiB each), q=3; step = one pass "
                                   "copy,scale,add,triad (4 launches)",
                       "n": n, "device": info["name"], "sm_count": info["sm_count"],
                       "l2": "inputs larger than L2 (3 x 1 GiB vs 126 MB): no flush",
                       "launch": tuned, "autotuned": bool(args.tune)},
            "kernels": kernels, "kernels_f32": kernels_f32, "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 4 * args.steps, "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    sx.sx_executor_destroy(e)
    sx.sx_target_destroy(t)
    if dist:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 27)
    ap.add_argument("--ref-n", type=int, default=1 << 22)
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--tune-cache", default="")
    ap.add_argument("--quick", action="store_true", help="FP64 pass only (no FP32, e2e, sections)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=1 << 24)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--sections", default="")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
