#!/usr/bin/env python
"""Benchmark of the STREAM hot path on B300 (Heller et al., Section 5, Listing 4).

One step = one STREAM pass (Copy c=a, Scale b=c*q, Add c=a+b, Triad a=b+c*q; q=3) over three
device-resident FP64 arrays of n = 2^27 elements (1 GiB each, far beyond the 126 MB L2, so no
L2 flush is needed between steps), seeded uniform in [-1, 1).  ``value`` is the STREAM byte
count of the pass (copy/scale 2*n*8 B, add/triad 3*n*8 B) over the device time, the slowest
rank's time taken for the job: by default summed over ranks (weak scaling: every rank runs
arrays of its own); with ``--shard`` each logical array is split into one contiguous block per
rank (Section 4.1's block allocator and co-located executor; strong scaling) and ``value`` is
the whole arrays' bytes over that time.  Either way there is no collective on the data path.

Also reported on the same JSON line: per-kernel GB/s (FP64 and FP32), the roofline of the
dominant kernel (Triad) against the measured HBM copy bandwidth, the end-to-end figure through
the C ABI from pinned host buffers, the CPU oracle on a bounded sample, SM clocks sampled during
the timed region, and the sections: "batched" (the persistent batched launcher vs one launch
per instance), "served" (the continuous-batching server vs a per-call FIFO), "small" (small
arrays: direct launches vs CUDA graphs vs one fused kernel), "overlap" (STREAM sets on one
stream vs one target and stream per set) and "copies" (host<->device copy bandwidth), plus the
oracle's loops block-partitioned over the host cores.  The batched and served sections appear
in full as "batched_detail" and "served_detail"; compact "batched" and "served" comparisons
(graph vs per-call, continuous vs FIFO: throughput, p50/p99) close the line.

``--impl reference`` times the CPU oracle (serial C, one core) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import itertools
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
RESEED_EVERY = 100

# dram__bytes_read.sum + dram__bytes_write.sum of one Triad launch (FP64, n = 2^27) from an ncu
# capture, with the sha256 of the kernel source it was taken on; reported as null when the
# source has changed since.
NCU_TRAFFIC = {"kernel": "k_stream_vec<3, double, 32, 2, 0, 4>", "n": 1 << 27,
               "bytes": 4 * 772062976,  # captured at n = 2^25 (536935680 read + 235127296 written), x4
               "cfg": {"variant": 1, "vec_bytes": 32, "unroll": 2, "cache_hint": 0, "fp64_mul": 2},
               "source_sha256": "5fe4c1bef26ab03dc7da71cae4893fc7c0c04ffe7a5bbffa481e703a2cfb3872"}


def _rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def job_throughput(dist, local_ms, bytes_per_step, steps, world, device, scaling="weak"):
    """Whole-job throughput (GB/s); the job's time is the slowest rank's (a MAX over ranks, the
    only collective).  weak: every rank moved `bytes_per_step` per step on arrays of its own, so
    the job moved `world` times that.  strong (the block partition): `bytes_per_step` is the
    whole logical array's, shared out over the ranks.  Returns (GB/s, max time in ms)."""
    ms = float(local_ms)
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    total = world * bytes_per_step if scaling == "weak" else bytes_per_step
    return total * steps / (ms * 1e-3) / 1e9, ms


def shard_block(sx, n, world, rank):
    """(offset, count) of this rank's contiguous block of one logical n-element array (Section
    4.1's block allocator over a vector of targets, one target per rank)."""
    return sx.sx_block_partition(n, world, rank)


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _kernel_source_sha():
    """sha256 over the sources of the pass kernels (vector kernels and their device helpers)."""
    h = hashlib.sha256()
    for name in ("sx_kernels.cu", "sx_device.cuh"):
        with open(os.path.join(ROOT, "paper_2206_06302_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


# NVML clock-event reason bits (nvmlClocksEventReason*) the bench reports by name
NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


def clock_summary(samples, window, max_mhz):
    """Summary of (time, SM MHz, reason bits) samples: those inside `window` (start, end), or all
    if none falls inside; the median SM clock and every reason seen active."""
    lo, hi = window
    inside = [x for x in samples if lo is not None and hi is not None and lo <= x[0] <= hi] or list(samples)
    if not inside:
        return None
    reasons = sorted({name for _, _, bits in inside for bit, name in NVML_REASONS.items() if bits & bit})
    return {"sm_mhz": statistics.median(m for _, m, _ in inside), "sm_max_mhz": max_mhz,
            "reasons": reasons, "samples": len(inside)}


class NvmlReader:
    """Reads (never sets) a GPU's SM clock, maximum SM clock and clock-event reasons through the
    driver's NVML library (libnvidia-ml.so.1) with ctypes.  The GPU is found by the UUID CUDA
    reports for `device` (NVML's indices need not follow CUDA's), else by index."""

    def __init__(self, lib, handle, reasons_fn):
        self.lib, self.h, self._reasons = lib, handle, reasons_fn

    @classmethod
    def open(cls, device):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            found = False
            try:
                import torch
                uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
                found = lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) == 0
            except Exception:  # noqa: BLE001 (no UUID from CUDA: by index)
                found = False
            if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device), ctypes.byref(h)) != 0:
                return None
            fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
            return cls(lib, h, fn)
        except (OSError, AttributeError):
            return None

    def _clock(self, getter):
        import ctypes
        v = ctypes.c_uint(0)
        if getter(self.h, ctypes.c_int(1), ctypes.byref(v)) != 0:  # 1: NVML_CLOCK_SM
            raise OSError("NVML clock query failed")
        return v.value

    def sm_mhz(self):
        return self._clock(self.lib.nvmlDeviceGetClockInfo)

    def sm_max_mhz(self):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def reasons(self):
        import ctypes
        v = ctypes.c_ulonglong(0)
        if self._reasons(self.h, ctypes.byref(v)) != 0:
            raise OSError("NVML reasons query failed")
        return v.value

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """SM clocks and throttle reasons during the timed region: NVML read every 2 ms by a thread
    (the samples between mark_start and mark_stop are summarised), and nvidia-smi every 100 ms
    beside it."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None
        self.nvml_samples, self.window, self.nvml_max = [], [None, None], None
        self._stop = False
        self._thread = None
        self._nvml = None

    def _poll_nvml(self, nvml):
        while not self._stop:
            try:
                self.nvml_samples.append((time.perf_counter(), nvml.sm_mhz(), nvml.reasons()))
            except OSError:  # a sample that fails is skipped
                pass
            time.sleep(0.002)

    def __enter__(self):
        nvml = self._nvml = NvmlReader.open(self.device)
        if nvml is not None:
            import threading
            self.nvml_max = nvml.sm_max_mhz()
            self._thread = threading.Thread(target=self._poll_nvml, args=(nvml,), daemon=True)
            self._thread.start()
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

    def mark_start(self):
        self.window[0] = time.perf_counter()

    def mark_stop(self):
        self.window[1] = time.perf_counter()

    def __exit__(self, *exc):
        self._stop = True
        if self._thread is not None:
            self._thread.join(timeout=1)
        if self._nvml is not None and (self._thread is None or not self._thread.is_alive()):
            self._nvml.close()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def smi_summary(self):
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

    def summary(self):
        """NVML's summary of the timed region (with nvidia-smi's beside it), or nvidia-smi's alone."""
        smi = self.smi_summary()
        nv = clock_summary(self.nvml_samples, self.window, self.nvml_max) if self.nvml_samples else None
        if nv is None:
            return smi
        nv["source"] = "NVML every 2 ms between the start and the end of the timed passes"
        if smi.get("reasons"):
            nv["reasons"] = sorted(set(nv["reasons"]) | {r for r in smi["reasons"] if "unavailable" not in r
                                                        and r != "no samples"})
        nv["smi"] = smi
        return nv


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
        "config": {"workload": f"STREAM F64 n=2^{args.n.bit_length() - 1} per array "
                               f"({args.n * 8 / 2 ** 30:g} GiB each), q={Q:g}; step = one pass "
                               "copy,scale,add,triad (4 launches)",
                   "n": args.n, "sample_n": n,
                   "sample": f"each step is the oracle's pass over n={n} per array, a bounded sample "
                             "of the workload; GB/s counts the sample's STREAM bytes"},
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"n={n} FP64 per array, {args.steps} passes", "cpu": _cpu_model()},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------
# GPU legs
# ----------------------------------------------------------------------------------------------

def stream_kernels(sx, torch, t, stream, e, dtype_code, n, steps, seed_instance, q=Q,
                   base_seed=None, init="uniform", doubling=False, index_base=0):
    """Arrays (constructed), pass sequence, a pass function and per-pass events of `steps` timed
    STREAM passes.  The caller runs its warm-up passes with the same function right before the
    timed ones, so that the timed region does not start on a GPU left idle by construction and
    set-up.  init "uniform": seeded values in [-1, 1); "closed-form": a = 1, b = 2, c = 0.
    doubling: a is doubled once after construction, as classic STREAM does before its timed
    loop.  index_base: generator index of element 0 (a block of a longer logical array)."""
    import stream_inputs as si
    base_seed = si.BASE_SEED if base_seed is None else base_seed
    es = 8 if dtype_code == sx.SX_F64 else 4
    arrs = [sx.sx_alloc(t, dtype_code, n) for _ in range(3)]
    a, b, c = arrs

    def construct():
        if init == "closed-form":
            for arr, v in zip(arrs, (1.0, 2.0, 0.0)):
                sx.sx_bulk_construct(arr, v)
        else:
            for k, arr in enumerate(arrs):
                sx.sx_seed_uniform_at(arr, si.array_seed(base_seed, k, seed_instance), -1.0, 1.0, index_base)
        if doubling:
            sx.sx_execute_async(e[sx.SX_OP_SCALE], sx.SX_OP_SCALE, a, None, a, 2.0, future=False)

    construct()
    seq = [("copy", sx.SX_OP_COPY, a, None, c), ("scale", sx.SX_OP_SCALE, c, None, b),
           ("add", sx.SX_OP_ADD, a, b, c), ("triad", sx.SX_OP_TRIAD, b, c, a)]
    count = [0]

    def one_pass(evs=None):
        # The workload is 100 passes from seeded inputs (|a| grows as 15^k: FP64 would reach
        # inf near k = 262).  Every 100 passes (warm-up passes included) the arrays are
        # constructed again, between the per-pass events, so it is not in the timed sum.
        if count[0] and count[0] % RESEED_EVERY == 0:
            construct()
        count[0] += 1
        if evs is not None:
            evs[0].record(stream)
        for k, (_, op, x, y, o) in enumerate(seq):
            sx.sx_execute_async(e[op], op, x, y, o, q, future=False)
            if evs is not None:
                evs[k + 1].record(stream)

    torch.cuda.synchronize()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    return arrs, seq, one_pass, events, es


def reseeds_between(first, count):
    """Constructions that passes number first .. first + count - 1 (from 0) start with: one
    before every pass whose number is a positive multiple of RESEED_EVERY."""
    return sum(1 for c in range(first, first + count) if c and c % RESEED_EVERY == 0)


def _pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(p / 100.0 * (len(xs) - 1)))))
    return xs[k]


def batched_section(sx, torch, t, stream, args, rank):
    """4096 independent FP64 triad/add instances, lengths log-uniform in [2^10, 2^22]: one
    persistent graph-captured launch (autotuned shape) vs one launch per instance.  The two
    launches' outputs are compared bit for bit on 8 instances (parity with the oracle is the
    tests' part), and those instances' inputs against the seeded generator."""
    import stream_inputs as si
    _, world, _ = _rank_env()
    if args.shard:
        # instances assigned whole to ranks: this rank's contiguous block of the one workload,
        # each instance seeded by its index in the whole list
        first, count = shard_block(sx, args.batch_count, world, rank)
        inst = si.batched_instances(si.BASE_SEED, args.batch_count)[first:first + count]
    else:
        first, inst = 0, si.batched_instances(si.BASE_SEED + rank, args.batch_count)
    offs, total = [], 0
    for _, n in inst:
        r = []
        for _ in range(3):
            total = (total + 255) // 256 * 256
            r.append(total)
            total += n * 8
        offs.append(r)
    buf = sx.sx_alloc(t, sx.SX_U8, total)
    base = sx.sx_array_data(buf)[0]
    seeds = []
    for k, (_, n) in enumerate(inst):
        for j in (0, 1):
            seeds.append(sx.sx_batch_item(op=sx.SX_OP_SEED, dtype=sx.SX_F64, n=n, out=base + offs[k][j],
                                          q=-1.0, q2=1.0, seed=si.array_seed(si.BASE_SEED, j, first + k)))
    sb = sx.sx_batch_create(t, seeds)
    sx.sx_batch_launch(sb)
    sx.sx_target_synchronize(t)
    sx.sx_batch_destroy(sb)
    code = {"add": sx.SX_OP_ADD, "triad": sx.SX_OP_TRIAD}
    items = [sx.sx_batch_item(op=code[op], dtype=sx.SX_F64, n=n, x=base + o[0], y=base + o[1],
                              out=base + o[2], q=Q) for (op, n), o in zip(inst, offs)]
    b = sx.sx_batch_create(t, items)
    best, _ = sx.sx_tune_batch(b)
    cfg, tiles, nbytes = sx.sx_batch_info(b)

    def timed(launch, reps):
        for _ in range(2):
            launch()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        for r in range(reps):
            ev[2 * r].record(stream)
            launch()
            ev[2 * r + 1].record(stream)
        torch.cuda.synchronize()
        return sorted(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(reps))

    g_ms = timed(lambda: sx.sx_batch_launch(b), args.batch_reps)
    p_ms = timed(lambda: sx.sx_batch_launch_percall(b), max(3, args.batch_reps // 2))
    # the same per-call launches captured once into a CUDA graph and replayed: one kernel node per
    # instance without the host's cost per launch, the strongest form of one launch per instance
    pcg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pcg, stream=stream, capture_error_mode="thread_local"):
        sx.sx_batch_launch_percall(b)

    def replay_percall():  # on the target's stream (a replay goes to torch's current stream)
        with torch.cuda.stream(stream):
            pcg.replay()

    pg_ms = timed(replay_percall, max(3, args.batch_reps // 2))
    # the same items through the entry point that allocates nothing (tiles of at least 1 MiB, so
    # the workload's tiles fit its static table): device time, and the host time of each call when
    # calls are enqueued back to back, beside that of a graph launch
    na_cfg = dict(cfg)
    na_cfg["chunk_bytes"] = max(cfg["chunk_bytes"], 1 << 20)
    na_ms = timed(lambda: sx.sx_batch_run_noalloc(stream.cuda_stream, items, na_cfg), max(3, args.batch_reps // 2))

    def host_us(call, reps):
        call()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            t0 = time.perf_counter()
            call()
            out.append((time.perf_counter() - t0) * 1e6)
        torch.cuda.synchronize()
        return sorted(out)

    na_host = host_us(lambda: sx.sx_batch_run_noalloc(stream.cuda_stream, items, na_cfg), 5)
    g_host = host_us(lambda: sx.sx_batch_launch(b), 5)
    sx.sx_batch_set_record(b, True)
    sx.sx_batch_launch(b)
    comp_g = [v / 1e6 for v in sx.sx_batch_completion_ns(b, len(items))]
    sx.sx_batch_launch_percall(b)
    comp_p = [v / 1e6 for v in sx.sx_batch_completion_ns(b, len(items))]
    sx.sx_batch_set_record(b, False)
    spot = list(range(0, len(items), max(1, len(items) // 8)))

    def snapshot(j):
        out = []
        for k in spot:
            n = inst[k][1]
            h = np.empty(n, np.float64)
            w = sx.sx_array_wrap(t, sx.SX_F64, base + offs[k][j], n)
            sx.sx_copy_d2h(h.ctypes.data, w, n)
            sx.sx_free(w)
            out.append(h.view(np.uint64))
        return out

    def poison():  # a sentinel in the sampled outputs, so that a launch that did not run shows
        for k in spot:
            w = sx.sx_array_wrap(t, sx.SX_F64, base + offs[k][2], inst[k][1])
            sx.sx_bulk_construct(w, -7.0)
            sx.sx_free(w)

    poison()
    sx.sx_batch_launch(b)
    sx.sx_target_synchronize(t)
    after_graph = snapshot(2)
    poison()
    sx.sx_batch_launch_percall(b)
    sx.sx_target_synchronize(t)
    after_percall = snapshot(2)
    poison()
    sx.sx_batch_run_noalloc(stream.cuda_stream, items, na_cfg)
    sx.sx_target_synchronize(t)
    after_noalloc = snapshot(2)
    poison()
    replay_percall()
    torch.cuda.synchronize()
    after_percall_graph = snapshot(2)
    del pcg
    same = all(np.array_equal(g, p) for g, p in zip(after_graph, after_percall)) and \
        all(np.array_equal(g, p) for g, p in zip(after_graph, after_percall_graph))
    same_noalloc = all(np.array_equal(g, p) for g, p in zip(after_graph, after_noalloc))
    inputs_ok = all(np.array_equal(h, si.uniform(si.array_seed(si.BASE_SEED, 0, first + k), inst[k][1], np.float64)
                                   .view(np.uint64)) for k, h in zip(spot, snapshot(0)))
    sx.sx_batch_destroy(b)
    sx.sx_free(buf)
    gm, pm, pgm = g_ms[len(g_ms) // 2], p_ms[len(p_ms) // 2], pg_ms[len(pg_ms) // 2]
    return {
        "share": (f"instances [{first}, {first + len(inst)}) of {args.batch_count}, assigned whole to this rank"
                  if args.shard else "all instances"),
        "workload": f"{len(items)} FP64 triad/add instances, n log-uniform in [2^10, 2^22] "
                    f"(seeded), {nbytes / 1e9:.1f} GB moved per launch",
        "tuned": cfg, "tiles": tiles,
        "graph_ms": round(gm, 4), "graph_GB/s": round(nbytes / (gm * 1e-3) / 1e9, 1),
        "graph_frac_measured": round(nbytes / (gm * 1e-3) / 1e9 / _measured_peaks()[0], 4),
        "percall_ms": round(pm, 4), "percall_GB/s": round(nbytes / (pm * 1e-3) / 1e9, 1),
        "speedup": round(pm / gm, 3),
        "percall_graph_ms": round(pgm, 4), "percall_graph_GB/s": round(nbytes / (pgm * 1e-3) / 1e9, 1),
        "speedup_vs_percall_graph": round(pgm / gm, 3),
        "completion_ms_p50": {"graph": round(_pct(comp_g, 50), 4), "percall": round(_pct(comp_p, 50), 4)},
        "completion_ms_p99": {"graph": round(_pct(comp_g, 99), 4), "percall": round(_pct(comp_p, 99), 4)},
        "launches": {"graph": 1, "percall": len(items), "percall_graph": f"1 graph of {len(items)} kernel nodes"},
        "graph_equals_percall_8_instances": same, "inputs_match_generator_8_instances": inputs_ok,
        "noalloc": {"what": "sx_batch_run_noalloc on the same items, calls enqueued back to back",
                    "cfg": na_cfg, "device_ms": round(na_ms[len(na_ms) // 2], 4),
                    "host_us_per_call_median": round(na_host[len(na_host) // 2], 1),
                    "graph_launch_host_us_median": round(g_host[len(g_host) // 2], 1),
                    "equals_graph_8_instances": same_noalloc},
    }


def batched_summary(b):
    """The batched comparison in a few hundred bytes: one graph launch vs one launch per instance
    (enqueued one by one, and replayed from a graph of per-instance kernel nodes: device time,
    STREAM bytes per second; per-instance completion p50/p99 of the first two) and whether the
    graph launch beats the per-call launches on throughput and on p99."""
    p50, p99 = b["completion_ms_p50"], b["completion_ms_p99"]
    return {"what": b["workload"],
            "ms": {"graph": b["graph_ms"], "percall": b["percall_ms"], "percall_graph": b.get("percall_graph_ms")},
            "GB/s": {"graph": b["graph_GB/s"], "percall": b["percall_GB/s"],
                     "percall_graph": b.get("percall_graph_GB/s")},
            "speedup": b["speedup"], "speedup_vs_percall_graph": b.get("speedup_vs_percall_graph"),
            "p50_ms": p50, "p99_ms": p99,
            "bit_identical_8_instances": b["graph_equals_percall_8_instances"],
            "noalloc_ms": b["noalloc"]["device_ms"],
            "noalloc_host_us_per_call": b["noalloc"]["host_us_per_call_median"],
            "graph_launch_host_us": b["noalloc"]["graph_launch_host_us_median"],
            "beats_percall": {"throughput": b["graph_GB/s"] > b["percall_GB/s"],
                              "throughput_vs_percall_graph": (b["graph_GB/s"] > b["percall_graph_GB/s"]
                                                              if b.get("percall_graph_GB/s") else None),
                              "p99": p99["graph"] < p99["percall"]}}


def served_load_medians(runs):
    """Per (offered load, mode): the median over the replays of p50, p99 and GB/s, and every
    replay's p99 beside it.  An occasional stall of the host (a thread that wakes late) shows in
    one replay's p99 and not in the median."""
    groups = {}
    for r in runs:
        groups.setdefault((r["offered_load"], r["mode"]), []).append(r)
    return {key: {"p50_ms": statistics.median(r["p50_ms"] for r in rs),
                  "p99_ms": statistics.median(r["p99_ms"] for r in rs),
                  "GB/s": statistics.median(r["GB/s"] for r in rs),
                  "p99_runs_ms": [r["p99_ms"] for r in rs]}
            for key, rs in groups.items()}


def served_summary(s):
    """The served comparison in a few hundred bytes: continuous batching vs the per-call FIFO at
    saturation (best run and every run) and, per offered load, [continuous, fifo] p50 / p99 and
    GB/s (medians over the replays, with every replay's p99); and whether continuous batching
    beats the FIFO on saturation throughput and on p99 at every load."""
    med = served_load_medians(s["runs"])
    loads = sorted({r["offered_load"] for r in s["runs"]})
    per = {}
    for ld in loads:
        c, f = med.get((ld, "continuous")), med.get((ld, "fifo"))
        if c and f:
            per[f"{ld:g}"] = {"p50_ms": [c["p50_ms"], f["p50_ms"]], "p99_ms": [c["p99_ms"], f["p99_ms"]],
                              "GB/s": [c["GB/s"], f["GB/s"]]}
            if len(c["p99_runs_ms"]) > 1 or len(f["p99_runs_ms"]) > 1:
                per[f"{ld:g}"]["p99_runs_ms"] = [c["p99_runs_ms"], f["p99_runs_ms"]]
    sat = s["saturation_GB/s"]
    return {"what": "continuous batching vs per-call FIFO; per load [continuous, fifo]; GB/s in STREAM bytes "
                    "(input construction and operation); continuous_split_phases: batching without the "
                    "construct-then-operate pieces; *_dram_*: the DRAM traffic each mode moves for that work "
                    "(continuous reads no input back)",
            "saturation_GB/s": sat, "saturation_runs_GB/s": s.get("saturation_runs_GB/s"),
            "saturation_frac_measured": s.get("saturation_frac_measured"),
            "saturation_dram_GB/s": s.get("saturation_dram_GB/s"),
            "saturation_dram_frac_measured": s.get("saturation_dram_frac_measured"),
            "saturation_gain": round(sat["continuous"] / sat["fifo"], 4) if sat.get("fifo") else None,
            "saturation_gain_worst_run": (round(min(s["saturation_runs_GB/s"]["continuous"]) /
                                                max(s["saturation_runs_GB/s"]["fifo"]), 4)
                                          if s.get("saturation_runs_GB/s") else None),
            "loads": per,
            "beats_fifo": {"throughput": sat["continuous"] > sat["fifo"],
                           "p99_every_load": all(v["p99_ms"][0] <= v["p99_ms"][1] for v in per.values())}}


def serve_run(sx, t, work, times, budget_bytes, mode, server_kw=None):
    """One replay of `work` arriving at `times` through a server in `mode`: latencies (ms) of the
    requests in order (None if rejected) and the server's statistics and makespan."""
    kw = dict(server_kw or {})
    s = sx.sx_server_create(t, budget_bytes=budget_bytes, mode=mode, **kw)
    ids = sx.sx_server_replay(s, work, times)
    lat, t0, t1 = [], None, None
    for rid in ids:
        st = sx.sx_server_wait(s, rid, 600000)
        if st["state"] == sx.SX_REQ_REJECTED:
            lat.append(None)
            continue
        lat.append((st["t_done"] - st["t_submit"]) * 1e3)
        t0 = st["t_submit"] if t0 is None else min(t0, st["t_submit"])
        t1 = st["t_done"] if t1 is None else max(t1, st["t_done"])
    stats = sx.sx_server_stats_get(s)
    sx.sx_server_destroy(s)
    return lat, stats, (t1 - t0) if t1 is not None else float("nan")


def shard_requests(reqs, world, rank):
    """A served request stream dealt out to `world` servers in turn (request k to rank k mod
    world), each keeping its requests' arrival times: every rank sees 1/world of the rate."""
    return [r for k, r in enumerate(reqs) if k % world == rank]


def served_workload(sx, seed, count, dram=None, world=1, rank=0):
    """The served requests (sx_request list), their element counts and STREAM byte counts (with
    world > 1: rank's share, shard_requests).  If `dram` is a dict, it receives the workload's
    total DRAM bytes under each mode: "continuous" (every piece stores x, y and out and reads
    nothing back) and "fifo" (the operation reads the inputs back from DRAM)."""
    import stream_inputs as si
    reqs = shard_requests(si.poisson_requests(seed, count, rate_per_s=1.0), world, rank)
    ops = {"copy": sx.SX_OP_COPY, "scale": sx.SX_OP_SCALE, "add": sx.SX_OP_ADD, "triad": sx.SX_OP_TRIAD}
    dts = {"f64": (sx.SX_F64, 8), "f32": (sx.SX_F32, 4)}
    work, nbytes = [], []
    written = read = 0
    for r in reqs:
        code, es = dts[r["dtype"]]
        two = r["op"] in ("add", "triad")
        # inputs construction (x, and y for add/triad) plus the operation itself
        nbytes.append(r["n"] * es * ((2 if two else 1) + (3 if two else 2)))
        written += r["n"] * es * ((2 if two else 1) + 1)
        read += r["n"] * es * (2 if two else 1)
        if dram is not None:
            dram["continuous"], dram["fifo"] = written, written + read
        work.append(sx.sx_request(op=ops[r["op"]], dtype=code, n=r["n"], q=Q,
                                  seed_x=si.word_scalar(r["seed"], 0), seed_y=si.word_scalar(r["seed"], 1),
                                  lo=-1.0, hi=1.0, flags=sx.SX_REQ_AUTO_RELEASE))
    return reqs, work, nbytes


def served_section(sx, torch, t, stream, args, rank):
    """Poisson stream of copy/scale/add/triad requests (FP64/FP32), n log-uniform in
    [2^12, 2^28], inputs constructed on the device, 64 GB arena.  After an untimed warm-up,
    both modes at saturation (every request at t=0; best of three runs each); the per-call FIFO's
    saturation throughput is the measured single-stream capacity.  Then continuous batching vs the per-call FIFO at offered
    loads of 0.5, 0.8 and 0.95 of that capacity, three replays each: p50/p99 latency (submission
    to completion seen by the server), the p99 of the shorter half of the requests, and
    throughput."""
    import stream_inputs as si
    dram = {}
    _, world, _ = _rank_env()
    if args.shard:  # one request stream dealt out to the ranks
        reqs, work, nbytes = served_workload(sx, si.BASE_SEED + 7, args.serve_count, dram, world, rank)
    else:
        reqs, work, nbytes = served_workload(sx, si.BASE_SEED + 7 + rank, args.serve_count, dram)
    mean_bytes = sum(nbytes) / len(nbytes)
    budget = int(args.serve_budget_gb * 1e9)
    median_n = sorted(r["n"] for r in reqs)[len(reqs) // 2]
    short = [k for k, r in enumerate(reqs) if r["n"] <= median_n]
    modes = ((sx.SX_SERVE_CONTINUOUS, "continuous"), (sx.SX_SERVE_FIFO, "fifo"))
    out = {"share": (f"requests k with k mod {world} = {rank} of {args.serve_count}" if args.shard else "all requests"),
           "workload": f"{len(reqs)} Poisson requests, ops uniform over copy/scale/add/triad, "
                       f"FP64/FP32 50/50, n log-uniform in [2^12, 2^28], inputs constructed on "
                       f"device, {args.serve_budget_gb:g} GB arena, mean {mean_bytes / 1e6:.1f} MB "
                       f"moved per request", "saturation_GB/s": {}, "runs": []}
    zero = [0.0] * len(work)
    # untimed warm-up of both modes (the first server of a process starts cold), then each mode
    # at saturation three times, alternating; the best run of each is its saturation throughput.
    # Beside them continuous batching with split_phases (inputs constructed in one piece, the
    # operation in a later one, reading them back from DRAM): what batching alone gives, without
    # the construct-then-operate pieces
    for mode, _ in modes:
        serve_run(sx, t, work[:200], zero[:200], budget, mode)
    sat_modes = ((sx.SX_SERVE_CONTINUOUS, "continuous", {}), (sx.SX_SERVE_CONTINUOUS, "continuous_split_phases",
                                                          {"split_phases": 1}), (sx.SX_SERVE_FIFO, "fifo", {}))
    sat = {name: [] for _, name, _ in sat_modes}
    for _ in range(3):
        for mode, name, kw in sat_modes:
            _, stats, span = serve_run(sx, t, work, zero, budget, mode, kw)
            sat[name].append(stats["bytes_moved"] / span / 1e9)
    for name, runs in sat.items():
        out["saturation_GB/s"][name] = round(max(runs), 1)
        out.setdefault("saturation_runs_GB/s", {})[name] = [round(v, 1) for v in runs]
        out.setdefault("saturation_frac_measured", {})[name] = round(max(runs) / _measured_peaks()[0], 4)
        # the DRAM traffic each mode has to move for the same work, at that rate (split phases: short
        # requests run fused and the others read their inputs back, between the two)
        if name in dram:
            out.setdefault("saturation_dram_GB/s", {})[name] = round(max(runs) * dram[name] / sum(nbytes), 1)
            out.setdefault("saturation_dram_frac_measured", {})[name] = round(
                max(runs) * dram[name] / sum(nbytes) / _measured_peaks()[0], 4)
    out["dram_bytes_per_stream_byte"] = {k: round(v / sum(nbytes), 4) for k, v in dram.items()}
    capacity = out["saturation_GB/s"]["fifo"] * 1e9
    out["capacity_from"] = "per-call FIFO throughput at saturation"
    # each offered load replayed --serve-load-reps times per mode, the modes alternating; the
    # summary takes the median of the replays
    for load in [float(v) for v in args.serve_loads.split(",") if v]:
        rate = load * capacity / mean_bytes
        times = [r["t"] / rate for r in reqs]
        for rep, (mode, name) in itertools.product(range(max(1, args.serve_load_reps)), modes):
            lat, stats, span = serve_run(sx, t, work, times, budget, mode)
            done = [v for v in lat if v is not None]
            out["runs"].append({
                "mode": name, "offered_load": load, "replay": rep, "rate_per_s": round(rate, 1),
                "p50_ms": round(_pct(done, 50), 4), "p99_ms": round(_pct(done, 99), 4),
                "p99_short_half_ms": round(_pct([lat[k] for k in short if lat[k] is not None], 99), 4),
                "mean_ms": round(sum(done) / len(done), 4),
                "GB/s": round(stats["bytes_moved"] / span / 1e9, 1),
                "launches": stats["launches"], "steps": stats["steps"],
                "rejected": len(lat) - len(done), "arena_peak_GB": round(stats["arena_peak"] / 1e9, 2)})
    return out


def dram_mix_section(sx, torch, t, stream, execs, n, reps=20):
    """The DRAM rate by read/write mix, with the library's own kernels on three FP64 arrays of n
    elements: sx_bulk_construct's fill (stores only), copy (one read per write) and add (two
    reads per write).  Each launch between its own CUDA events on the launching stream; the
    median of `reps` after 3 untimed ones.  Copy's rate is bounded by the DRAM's mixed-direction
    rate, which this shows beside the store-only rate."""
    arrs = [sx.sx_alloc(t, sx.SX_F64, n) for _ in range(3)]
    for k, a in enumerate(arrs):
        sx.sx_seed_uniform(a, k + 1, -1.0, 1.0)
    x, y, o = arrs

    def median_ms(fn):
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sorted(a.elapsed_time(b) for a, b in ev)[reps // 2]

    ms = {"fill": median_ms(lambda: sx.sx_bulk_construct(o, 1.5)),
          "copy": median_ms(lambda: sx.sx_execute_async(execs[sx.SX_OP_COPY], sx.SX_OP_COPY, x, None, o, Q, future=False)),
          "add": median_ms(lambda: sx.sx_execute_async(execs[sx.SX_OP_ADD], sx.SX_OP_ADD, x, y, o, Q, future=False))}
    for a in arrs:
        sx.sx_free(a)
    nb = n * 8
    return {"what": f"FP64 arrays of n={n}; median per-launch device time of {reps}",
            "fill_stores_only_GB/s": round(nb / (ms["fill"] * 1e-3) / 1e9, 1),
            "copy_1_read_1_write_GB/s": round(2 * nb / (ms["copy"] * 1e-3) / 1e9, 1),
            "add_2_reads_1_write_GB/s": round(3 * nb / (ms["add"] * 1e-3) / 1e9, 1)}


def fused_section(sx, torch, t, stream, n, rank, passes=100):
    """The workload's 100 FP64 passes as 4 launches per pass (replayed from the executor's
    captured graphs, after an untimed warm-up call that captures them) vs one fused kernel (the
    same roundings per element; bit-identical results, checked here on the whole arrays)."""
    import stream_inputs as si
    arrs = {tag: [sx.sx_alloc(t, sx.SX_F64, n) for _ in range(3)] for tag in ("iter", "fused")}

    def seed_all():
        for tag in arrs:
            for k, arr in enumerate(arrs[tag]):
                sx.sx_seed_uniform(arr, si.array_seed(si.BASE_SEED, k, rank), -1.0, 1.0)

    e = sx.sx_executor_create(t, sx.SX_PAR_TASK)
    # untimed warm-up of both forms (the first call captures the pass graphs), then the same
    # start values again
    seed_all()
    sx.sx_stream_iter(e, *arrs["iter"], Q, passes)
    sx.sx_stream_fused(e, *arrs["fused"], Q, passes)
    seed_all()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    sx.sx_stream_iter(e, *arrs["iter"], Q, passes)
    ev[1].record(stream)
    ev[2].record(stream)
    sx.sx_stream_fused(e, *arrs["fused"], Q, passes)
    ev[3].record(stream)
    torch.cuda.synchronize()
    t_iter, t_fused = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    same = True
    for a1, a2 in zip(arrs["iter"], arrs["fused"]):
        h1, h2 = np.empty(n, np.float64), np.empty(n, np.float64)
        sx.sx_copy_d2h(h1.ctypes.data, a1, n)
        sx.sx_copy_d2h(h2.ctypes.data, a2, n)
        same &= bool(np.array_equal(h1.view(np.uint64), h2.view(np.uint64)))
    for tag in arrs:
        for arr in arrs[tag]:
            sx.sx_free(arr)
    sx.sx_executor_destroy(e)
    stream_bytes = 10.0 * n * 8 * passes
    return {"passes": passes, "four_launches_ms": round(t_iter, 3), "fused_ms": round(t_fused, 3),
            "speedup": round(t_iter / t_fused, 3),
            "four_launches_GB/s": round(stream_bytes / (t_iter * 1e-3) / 1e9, 1),
            "fused_STREAM-equivalent_GB/s": round(stream_bytes / (t_fused * 1e-3) / 1e9, 1),
            "fused_dram_bytes": 4 * n * 8, "bit_identical": same}


def small_n_section(sx, torch, device=0, passes=100, sizes=(1 << 10, 1 << 14, 1 << 16, 1 << 18, 1 << 20, 1 << 22)):
    """Small arrays, where a STREAM pass is bound by the cost of its four kernel launches (the
    paper's small-size overhead): `passes` passes as `passes` single-pass calls (direct
    launches), as one sx_stream_iter call (replayed from CUDA graphs), and fused into one kernel.
    PAR_TASK executor on a target of its own, host clock from the first call to the wait (the
    graph is captured by an untimed warm-up call); FP64; the three modes' results are compared
    bit for bit (parity with the oracle is the tests' part)."""
    import stream_inputs as si
    tt = sx.sx_target_create(device)
    e = sx.sx_executor_create(tt, sx.SX_PAR_TASK)
    rows = []
    for n in sizes:
        host = si.stream_arrays(n, np.float64, base_seed=55)
        arrs = [sx.sx_alloc(tt, sx.SX_F64, n) for _ in range(3)]

        def load():
            for h, d in zip(host, arrs):
                sx.sx_copy_h2d(d, h.ctypes.data, n)
            sx.sx_target_synchronize(tt)

        def timed(fn):
            load()
            t0 = time.perf_counter()
            fn()
            sx.sx_executor_wait(e)
            return time.perf_counter() - t0

        def direct():
            for _ in range(passes):
                sx.sx_stream_iter(e, *arrs, Q, 1)

        modes = {"direct": direct, "graphs": lambda: sx.sx_stream_iter(e, *arrs, Q, passes),
                 "fused": lambda: sx.sx_stream_fused(e, *arrs, Q, passes)}
        res, results = {}, []
        for name, fn in modes.items():
            timed(fn)  # warm (captures the graphs)
            res[name] = min(timed(fn) for _ in range(3))
            got = [np.empty(n, np.float64) for _ in arrs]
            for d, g in zip(arrs, got):
                sx.sx_copy_d2h(g.ctypes.data, d, n)
            results.append(np.concatenate(got).view(np.uint64))
        same = all(np.array_equal(results[0], r) for r in results[1:])
        moved = 10.0 * n * 8 * passes
        rows.append({"n": n, **{f"{k}_us_per_pass": round(v * 1e6 / passes, 2) for k, v in res.items()},
                     **{f"{k}_GB/s": round(moved / v / 1e9, 1) for k, v in res.items()},
                     "modes_bit_identical": same})
        for d in arrs:
            sx.sx_free(d)
    sx.sx_executor_destroy(e)
    sx.sx_target_destroy(tt)
    return {"what": f"FP64 STREAM, {passes} passes: {passes} single-pass calls (4 launches each) vs one "
                    "call (CUDA graphs of 16 passes) vs one fused kernel; PAR_TASK, host clock incl. enqueue",
            "runs": rows}


def overlap_section(sx, torch, device=0, sets=4, passes=20, sizes=(1 << 16, 1 << 18, 1 << 20, 1 << 22, 1 << 24)):
    """Asynchronous execution over several targets (Section 3.3 async_execute/bulk_async_execute,
    Section 4.2: a target is a device and a stream).  `sets` independent FP64 STREAM array sets,
    `passes` passes each (one sx_stream_iter call per set, replayed from CUDA graphs), enqueued with
    PAR_TASK executors and waited for at the end: either every set on one target (one stream: the
    sets run one after another) or each set on a target of its own (one stream each, free to
    overlap).  Same memory in both modes (the one-stream mode borrows the sets' arrays).  Host clock
    from the first enqueue to the last wait (graphs captured by untimed warm-up runs); the two
    modes' results are compared bit for bit (parity with the oracle is the tests' part)."""
    import stream_inputs as si
    tgts = [sx.sx_target_create(device) for _ in range(sets)]
    execs = [sx.sx_executor_create(tt, sx.SX_PAR_TASK) for tt in tgts]
    rows = []
    for n in sizes:
        owned = [[sx.sx_alloc(tgts[k], sx.SX_F64, n) for _ in range(3)] for k in range(sets)]
        borrowed = [[sx.sx_array_wrap(tgts[0], sx.SX_F64, sx.sx_array_data(a)[0], n) for a in owned[k]]
                    for k in range(sets)]

        def seed():
            for k in range(sets):
                for j, a in enumerate(owned[k]):
                    sx.sx_seed_uniform(a, si.array_seed(si.BASE_SEED + 17, j, k), -1.0, 1.0)
            for tt in tgts:
                sx.sx_target_synchronize(tt)

        def run(concurrent):
            seed()
            t0 = time.perf_counter()
            for k in range(sets):
                if concurrent:
                    sx.sx_stream_iter(execs[k], *owned[k], Q, passes)
                else:
                    sx.sx_stream_iter(execs[0], *borrowed[k], Q, passes)
            for ex in execs:
                sx.sx_executor_wait(ex)
            return time.perf_counter() - t0

        def results():
            out = []
            for k in range(sets):
                for j in range(3):
                    got = np.empty(n, np.float64)
                    sx.sx_copy_d2h(got.ctypes.data, owned[k][j], n)
                    out.append(got.view(np.uint64))
            return out

        run(False)
        run(True)  # warm both
        one = min(run(False) for _ in range(3))
        first = results()
        many = min(run(True) for _ in range(3))
        same = all(np.array_equal(a, b) for a, b in zip(first, results()))
        moved = 10.0 * n * 8 * passes * sets
        rows.append({"n": n, "one_stream_ms": round(one * 1e3, 3), "stream_per_set_ms": round(many * 1e3, 3),
                     "speedup": round(one / many, 3), "one_stream_GB/s": round(moved / one / 1e9, 1),
                     "stream_per_set_GB/s": round(moved / many / 1e9, 1), "modes_bit_identical": same})
        for k in range(sets):
            for a in borrowed[k] + owned[k]:
                sx.sx_free(a)
    for ex in execs:
        sx.sx_executor_destroy(ex)
    for tt in tgts:
        sx.sx_target_destroy(tt)
    return {"what": f"{sets} independent FP64 STREAM sets x {passes} passes (one call per set, CUDA graphs), "
                    "PAR_TASK; one target (one stream) vs one target per set; host clock incl. enqueue",
            "runs": rows}


def copies_section(sx, torch, t, device=0, sizes=(1 << 20, 1 << 24, 1 << 28, 1 << 30), reps=5):
    """Host<->device copy algorithm (Section 4.2: copy between host and device is a CUDA memcpy)
    through sx_copy_h2d / sx_copy_d2h on pinned and pageable host buffers, and both directions at
    once (pinned; the two copies on two targets' streams).  Best of `reps`, host clock."""
    rows = []
    t2 = sx.sx_target_create(device)
    for nbytes in sizes:
        d1, d2 = sx.sx_alloc(t, sx.SX_U8, nbytes), sx.sx_alloc(t2, sx.SX_U8, nbytes)
        pin1 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        pin2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        page = np.ones(nbytes, np.uint8)

        def best(fn):
            fn()
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                fn()
                ts.append(time.perf_counter() - t0)
            return min(ts)

        def both():
            sx.sx_copy_h2d_async(d1, pin1.data_ptr(), nbytes)
            sx.sx_copy_d2h_async(pin2.data_ptr(), d2, nbytes)
            sx.sx_target_synchronize(t)
            sx.sx_target_synchronize(t2)

        r = {"bytes": nbytes,
             "h2d_pinned_GB/s": nbytes / best(lambda: sx.sx_copy_h2d(d1, pin1.data_ptr(), nbytes)) / 1e9,
             "d2h_pinned_GB/s": nbytes / best(lambda: sx.sx_copy_d2h(pin1.data_ptr(), d1, nbytes)) / 1e9,
             "h2d_pageable_GB/s": nbytes / best(lambda: sx.sx_copy_h2d(d1, page.ctypes.data, nbytes)) / 1e9,
             "d2h_pageable_GB/s": nbytes / best(lambda: sx.sx_copy_d2h(page.ctypes.data, d1, nbytes)) / 1e9,
             "both_directions_pinned_GB/s": 2 * nbytes / best(both) / 1e9}
        rows.append({k: (round(v, 2) if isinstance(v, float) else v) for k, v in r.items()})
        sx.sx_free(d1)
        sx.sx_free(d2)
        del pin1, pin2, page
    sx.sx_target_destroy(t2)
    return {"what": "sx_copy_h2d/d2h (synchronous) from pinned and pageable host memory; both directions "
                    "at once on two streams (pinned); best of %d, host clock" % reps, "runs": rows}


def _cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo), for the CPU baselines."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def cpu_oracle_threads_gbs(n: int, seconds: float):
    """The oracle's STREAM pass with its loops block-partitioned over the host cores: thread k
    runs the oracle on elements [n k / T, n (k + 1) / T) of each array, pinned to one core; a pass
    ends when every block has finished (every element's pass is independent of the others')."""
    import threading
    import oracle
    import stream_inputs as si
    cpus = sorted(os.sched_getaffinity(0))
    nt = len(cpus)
    a, b, c = si.stream_arrays(n, np.float64)
    oracle.default()
    bounds = [(n * k // nt, n * (k + 1) // nt) for k in range(nt)]
    start, end = threading.Barrier(nt + 1), threading.Barrier(nt + 1)
    stop = [False]

    def worker(k):
        os.sched_setaffinity(0, {cpus[k]})
        lo, hi = bounds[k]
        while True:
            start.wait()
            if stop[0]:
                return
            oracle.stream(a[lo:hi], b[lo:hi], c[lo:hi], Q, 1)
            end.wait()

    ths = [threading.Thread(target=worker, args=(k,), daemon=True) for k in range(nt)]
    for th in ths:
        th.start()
    start.wait()
    end.wait()  # warm (page in)
    passes, t0 = 0, time.perf_counter()
    while True:
        start.wait()
        end.wait()
        passes += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    stop[0] = True
    start.wait()
    for th in ths:
        th.join()
    return 10.0 * n * 8 * passes / el / 1e9, passes, el, nt


def graph_launch_ms(sx, torch, stream, e, op, x, y, o, launches=20, replays=5):
    """Device time per launch of `launches` back-to-back launches captured into one CUDA graph on
    `stream` (the target's stream), the median over `replays` replays after one untimed replay."""
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
        for _ in range(launches):
            sx.sx_execute_async(e, op, x, y, o, Q, future=False)
    with torch.cuda.stream(stream):
        g.replay()
        ts = []
        for _ in range(replays):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b) / launches)
    del g
    return sorted(ts)[replays // 2]


def run_sweep(args):
    """Size sweep (the paper's array-size figure): n = 2^lo..2^hi per array, FP64 and FP32, the
    four kernels, VECTOR vs BULK (TMA bulk-copy staging of the inputs) vs TMA (bulk copies both
    ways) vs TMA_TENSOR (the same with 2-D tensor-map copies) at fixed launch shapes.  Prints one
    JSON line.  Back-to-back launches on the same arrays: below ~2^22-2^23 elements the three
    arrays stay in the 126 MB L2."""
    import torch
    import paper_2206_06302_b300 as sx
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    t = sx.target_on_torch_stream(0, stream)
    shapes = {
        "vector": dict(variant=sx.SX_VARIANT_VECTOR, threads=256, vec_bytes=32, unroll=2, fp64_mul=2),
        "bulk": dict(variant=sx.SX_VARIANT_BULK, threads=256, blocks_per_sm=2, tile_bytes=16384,
                     stages=3, fp64_mul=2),
        "tma": dict(variant=sx.SX_VARIANT_TMA, threads=256, blocks_per_sm=2, tile_bytes=16384,
                    stages=3, fp64_mul=2),
        "tma_tensor": dict(variant=sx.SX_VARIANT_TMA_TENSOR, threads=256, blocks_per_sm=2,
                           tile_bytes=16384, stages=3, fp64_mul=2),
    }
    execs = {k: sx.sx_executor_create(t, sx.SX_PAR_TASK, v) for k, v in shapes.items()}
    l2 = sx.sx_target_info_get(t)["l2_bytes"]  # the regime split: the kernel's arrays fit in L2 or not
    ops = (("copy", sx.SX_OP_COPY, 2), ("scale", sx.SX_OP_SCALE, 2), ("add", sx.SX_OP_ADD, 3),
           ("triad", sx.SX_OP_TRIAD, 3))
    rows = []
    for dcode, dname, es in ((sx.SX_F64, "f64", 8), (sx.SX_F32, "f32", 4)):
        nmax = 1 << args.sweep_hi
        arrs = [sx.sx_alloc(t, dcode, nmax) for _ in range(3)]
        for k, arr in enumerate(arrs):
            sx.sx_seed_uniform(arr, k + 1, -1.0, 1.0)
        base = [sx.sx_array_data(a)[0] for a in arrs]
        for lg in range(args.sweep_lo, args.sweep_hi + 1):
            n = 1 << lg
            views = [sx.sx_array_wrap(t, dcode, p, n) for p in base]
            x, y, o = views
            for name, op, narr in ops:
                for vname, e in execs.items():
                    nbytes = narr * n * es
                    reps = int(min(2000, max(20, 4e-3 / max(nbytes / 6e12, 2e-6))))  # >= 20 timed launches per point
                    for _ in range(3):
                        sx.sx_execute_async(e, op, x, y, o, Q, future=False)
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(stream)
                    for _ in range(reps):
                        sx.sx_execute_async(e, op, x, y, o, Q, future=False)
                    ev1.record(stream)
                    ev1.synchronize()
                    ms = ev0.elapsed_time(ev1) / reps
                    row = {"dtype": dname, "log2n": lg, "op": name, "variant": vname,
                           "regime": "L2-resident" if nbytes <= l2 else "HBM",
                           "us": round(ms * 1e3, 2), "GB/s": round(nbytes / (ms * 1e-3) / 1e9, 1)}
                    if nbytes <= l2:
                        # the same launches captured once into a CUDA graph and replayed: the host's
                        # launch cost drops out, which bounds these sizes when launched one by one
                        gms = graph_launch_ms(sx, torch, stream, e, op, x, y, o)
                        row.update({"graph_us": round(gms * 1e3, 2), "graph_GB/s": round(nbytes / (gms * 1e-3) / 1e9, 1)})
                    rows.append(row)
            for v in views:
                sx.sx_free(v)
        for a in arrs:
            sx.sx_free(a)
    sx.sx_target_synchronize(t)
    print(json.dumps({"sweep": rows, "shapes": shapes, "l2_bytes": l2,
                      "note": "per-launch device time, back-to-back launches on the same arrays; "
                              "regime: the kernel's arrays together fit in L2 or not; graph_*: the same "
                              "launches replayed from a CUDA graph (L2-resident rows)"}),
          flush=True)
    return 0


def run_dram_mix(args):
    """The DRAM mix on its own, in a fresh process (see dram_mix_section): one JSON line.  The
    FP64 launch shapes are the tuner table's for --n."""
    import torch
    import paper_2206_06302_b300 as sx
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    t = sx.target_on_torch_stream(0, stream)
    e_auto = sx.sx_executor_create(t, sx.SX_PAR_TASK)
    execs = {op: sx.sx_executor_create(t, sx.SX_PAR_TASK, sx.sx_executor_resolve(e_auto, op, sx.SX_F64, args.n))
             for op in (sx.SX_OP_COPY, sx.SX_OP_ADD)}
    out = dram_mix_section(sx, torch, t, stream, execs, args.n)
    out["device"] = sx.sx_target_info_get(t)["name"]
    print(json.dumps({"dram_mix": out}), flush=True)
    for e in list(execs.values()) + [e_auto]:
        sx.sx_executor_destroy(e)
    sx.sx_target_destroy(t)
    return 0


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
    # --shard: one logical array of n elements per STREAM array, split into contiguous blocks, one
    # per rank (strong scaling); otherwise every rank runs whole arrays of its own (weak scaling)
    scaling = "strong" if args.shard else "weak"
    off, n_local = shard_block(sx, n, world, rank) if args.shard else (0, n)
    tune_n = args.tune_n or max(1, n_local)  # the size whose launch shapes the pass kernels use
    names = (("copy", sx.SX_OP_COPY), ("scale", sx.SX_OP_SCALE), ("add", sx.SX_OP_ADD),
             ("triad", sx.SX_OP_TRIAD))
    tuned = {}
    # the autotuner's table: the committed one for this device, then --tune-cache on top of it
    for path in (args.tune_table, args.tune_cache):
        if path and os.path.exists(path):
            sx.sx_tune_load(path)
    if args.tune:
        for dcode in (sx.SX_F64, sx.SX_F32):
            searched = False
            for name, op in names:
                if args.retune or sx.sx_tune_lookup(t, op, dcode, tune_n) is None:
                    sx.sx_tune(t, op, dcode, tune_n)
                    searched = True
            if searched:  # then the four kernels together, in the pass they run in
                sx.sx_tune_pass(t, dcode, tune_n)
        if args.tune_cache:
            sx.sx_tune_save(args.tune_cache)
    # a forced family takes its default shape, with half of the FP64 products on the integer units
    # as the tuned shapes have them (ignored for FP32 and for copy and add)
    forced = {"vector": dict(variant=sx.SX_VARIANT_VECTOR, fp64_mul=2),
              "bulk": dict(variant=sx.SX_VARIANT_BULK, fp64_mul=2),
              "tma": dict(variant=sx.SX_VARIANT_TMA, fp64_mul=2),
              "tma_tensor": dict(variant=sx.SX_VARIANT_TMA_TENSOR, fp64_mul=2)}
    e_auto = sx.sx_executor_create(t, sx.SX_PAR_TASK, forced.get(args.variant))
    execs = {}  # per dtype and op: an executor fixed to the shape resolved at tune_n
    for dcode, dname in ((sx.SX_F64, "f64"), (sx.SX_F32, "f32")):
        tuned[dname] = {name: sx.sx_executor_resolve(e_auto, op, dcode, tune_n) for name, op in names}
        execs[dcode] = {op: sx.sx_executor_create(t, sx.SX_PAR_TASK, tuned[dname][name])
                        for name, op in names}
    e = e_auto
    main_code, main_name = (sx.SX_F32, "f32") if args.dtype == "f32" else (sx.SX_F64, "f64")
    q = args.q

    peak, peak_kind = _measured_peaks()
    out = {}

    # ---- the timed region: STREAM passes (FP64 unless --dtype f32) ---------------------------
    instance = 0 if args.shard else rank  # blocks of one logical array share its seeds
    arrs, seq, one_pass, events, es = stream_kernels(
        sx, torch, t, stream, execs[main_code], main_code, n_local, args.steps, instance, q,
        args.seed, args.init, args.stream_doubling, index_base=off)
    with ClockSampler(local) as clocks:
        for _ in range(args.warmup):
            one_pass()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks.mark_start()
        for s in range(args.steps):
            one_pass(events[s])
        torch.cuda.synchronize()
        clocks.mark_stop()
    if dist:
        dist.barrier()
    sx.sx_target_synchronize(t)  # surfaces any device-side error word
    per = {name: 0.0 for name, *_ in seq}
    each = {name: [] for name, *_ in seq}  # per-pass times, for STREAM's min/avg/max report
    for s in range(args.steps):
        for k, (name, *_r) in enumerate(seq):
            ms_k = events[s][k].elapsed_time(events[s][k + 1])
            per[name] += ms_k
            each[name].append(ms_k)
    # sum of the passes' own device times (re-construction every 100 passes falls between them)
    total_ms = sum(events[s][0].elapsed_time(events[s][4]) for s in range(args.steps))
    step_bytes = 10.0 * n * es  # the whole logical arrays (shard) or one rank's arrays (weak)
    value, total_ms = job_throughput(dist, total_ms, step_bytes, args.steps, world, "cuda", scaling)
    bytes_per = {"copy": 2, "scale": 2, "add": 3, "triad": 3}
    kernels = {}
    for name in per:
        ms = per[name] / args.steps
        gbs = bytes_per[name] * n_local * es / (ms * 1e-3) / 1e9
        # STREAM's own convention besides the mean: the best pass, excluding the first
        rest = each[name][1:] or each[name]
        kernels[name] = {"ms": round(ms, 5), "GB/s": round(gbs, 1),
                         "frac_measured": round(gbs / peak, 4),
                         "frac_nominal_8TBs": round(gbs / NOMINAL_HBM_GBS, 4),
                         "ms_min_avg_max": [round(min(rest), 5), round(sum(rest) / len(rest), 5), round(max(rest), 5)],
                         "GB/s_best": round(bytes_per[name] * n_local * es / (min(rest) * 1e-3) / 1e9, 1)}
    clk = clocks.summary()

    # ---- FP32 per-kernel figures (same shape, fewer steps) -----------------------------------
    kernels_f32 = None
    if not args.quick and main_code == sx.SX_F64:
        for arr in arrs:
            sx.sx_free(arr)
        steps32 = max(3, min(args.steps, 200))
        arrs, seq, one_pass, ev32, es32 = stream_kernels(
            sx, torch, t, stream, execs[sx.SX_F32], sx.SX_F32, n_local, steps32, instance, q,
            args.seed, args.init, args.stream_doubling, index_base=off)
        for _ in range(args.warmup):
            one_pass()
        for s in range(steps32):
            one_pass(ev32[s])
        torch.cuda.synchronize()
        kernels_f32 = {}
        for k, (name, *_r) in enumerate(seq):
            ms = sum(ev32[s][k].elapsed_time(ev32[s][k + 1]) for s in range(steps32)) / steps32
            gbs = bytes_per[name] * n_local * es32 / (ms * 1e-3) / 1e9
            kernels_f32[name] = {"ms": round(ms, 5), "GB/s": round(gbs, 1),
                                 "frac_measured": round(gbs / peak, 4)}
    for arr in arrs:
        sx.sx_free(arr)

    # ---- end to end through the C ABI from pinned host buffers --------------------------------
    e2e = None
    if not args.quick and args.e2e_steps > 0:
        import stream_inputs as si
        host = []
        tdt, ndt = (torch.float32, np.float32) if main_code == sx.SX_F32 else (torch.float64, np.float64)
        for k in range(3):
            h = torch.empty(n_local, dtype=tdt, pin_memory=True)
            h.numpy()[:] = si.uniform(si.array_seed(si.BASE_SEED if args.seed is None else args.seed, k, instance),
                                      n_local, ndt, start=off) if k == 0 else 0.0
            host.append(h)
        dev = [sx.sx_alloc(t, main_code, n_local) for _ in range(3)]
        esync = sx.sx_executor_create(t, sx.SX_PAR, forced.get(args.variant))
        sx.sx_stream_host(esync, *(h.data_ptr() for h in host), *dev, q, 1)  # warm
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sx.sx_stream_host(esync, *(h.data_ptr() for h in host), *dev, q, 1)
        el = time.perf_counter() - t0
        e2e_gbs, el_ms = job_throughput(dist, el * 1e3, step_bytes, args.e2e_steps, world, "cuda", scaling)
        e2e = {"value": round(e2e_gbs, 2), "unit": "GB/s",
               "h2d_bytes_per_step": n_local * es, "d2h_bytes_per_step": 3 * n_local * es,
               "steps": args.e2e_steps,
               "what": "sx_stream_host: h2d a (a pass writes b and c before reading them) + one pass + "
                       "d2h a,b,c from pinned host memory, pipelined in 32 MiB chunks over 3 streams; host clock"}
        for d in dev:
            sx.sx_free(d)
        sx.sx_executor_destroy(esync)
        del host

    # ---- sections beyond the plain pass --------------------------------------------------------
    extra = {}
    if not args.quick and "batched" in args.sections:
        extra["batched"] = batched_section(sx, torch, t, stream, args, rank)
    if not args.quick and "served" in args.sections:
        extra["served"] = served_section(sx, torch, t, stream, args, rank)

    if not args.quick:
        extra["fused_100_passes"] = fused_section(sx, torch, t, stream, n, rank)
    if not args.quick and "small" in args.sections:
        extra["small_n_passes"] = small_n_section(sx, torch, local)
    if not args.quick and "overlap" in args.sections:
        extra["overlap_targets"] = overlap_section(sx, torch, local)
    if not args.quick and "copies" in args.sections:
        extra["copies"] = copies_section(sx, torch, t, local)

    # ---- CPU oracle on a bounded sample (rank 0, N=1 only) ------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        gbs, passes, el = cpu_oracle_gbs(args.cpu_n, args.cpu_seconds)
        cpu = {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"STREAM FP64 pass on n={args.cpu_n} per array, {passes} passes "
                         f"in {el:.1f} s (serial C, -O2 -ffp-contract=off)", "cpu": _cpu_model()}
        if args.cpu_threads_n:
            gbs, passes, el, nt = cpu_oracle_threads_gbs(args.cpu_threads_n, args.cpu_seconds / 2)
            extra["cpu_baseline_threads"] = {
                "value": round(gbs, 3), "unit": "GB/s", "cores": nt, "kind": "oracle loops, block-partitioned",
                "sample": f"STREAM FP64 pass on n={args.cpu_threads_n} per array, {passes} passes in "
                          f"{el:.1f} s, one contiguous block per pinned thread", "cpu": _cpu_model()}

    triad_ms = per["triad"] / args.steps
    achieved = 3 * n_local * es / (triad_ms * 1e-3) / 1e9
    traffic = None
    # the captured traffic holds for the captured case only: FP64, q = 3, this n and launch shape
    same_kernel = main_code == sx.SX_F64 and q == Q and \
        all(tuned["f64"]["triad"].get(k) == v for k, v in NCU_TRAFFIC["cfg"].items())
    if NCU_TRAFFIC["bytes"] and NCU_TRAFFIC["source_sha256"] == _kernel_source_sha() \
            and NCU_TRAFFIC["n"] == n_local and same_kernel:
        traffic = NCU_TRAFFIC["bytes"]
    roofline = {"bound": "hbm", "kernel": f"triad {main_name}", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "frac_nominal_8TBs": round(achieved / NOMINAL_HBM_GBS, 4),
                "algorithmic_bytes_per_launch": 3 * n_local * es, "traffic": traffic}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 5),
            "higher_is_better": True, "scaling": scaling, "vs_baseline": None, "dtype": main_name,
            "data": ("synthetic: a=1, b=2, c=0" if args.init == "closed-form" else
                     "synthetic: seeded SplitMix64 uniform [-1,1)") + ", constructed on the device" +
                    (", a doubled once" if args.stream_doubling else ""),
            "config": {"workload": f"STREAM {main_name.upper()} n=2^{n.bit_length() - 1} per array "
                                   f"({n * es / 2 ** 30:g} GiB each), q={q:g}; step = one pass "
                                   "copy,scale,add,triad (4 launches)",
                       "n": n, "device": info["name"], "sm_count": info["sm_count"],
                       "l2": ("inputs larger than L2: no flush" if 3 * n_local * es > info["l2_bytes"] else
                              "inputs fit in L2 (L2-resident regime)"),
                       "parallelism": (f"block partition of each array over {world} rank(s); rank 0 holds "
                                       f"[{off}, {off + n_local})" if args.shard else
                                       f"{world} replica(s), arrays of their own"),
                       "variant": args.variant, "init": args.init, "stream_doubling": args.stream_doubling,
                       "launch": tuned, "autotuned": bool(args.tune)},
            "kernels": kernels, "kernels_f32": kernels_f32, "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 4 * args.steps + (3 + int(args.stream_doubling)) * reseeds_between(args.warmup, args.steps),
            "clocks": clk,
        }
        # the verbose sections first; the compact batched and served comparisons close the line,
        # so that a reader of its last few kilobytes still sees them
        for k, v in extra.items():
            if k in ("batched", "served"):
                line[k + "_detail"] = v
            else:
                line[k] = v
        if "batched" in extra:
            line["batched"] = batched_summary(extra["batched"])
        if "served" in extra:
            line["served"] = served_summary(extra["served"])
        print(json.dumps(line), flush=True)
    for d in execs.values():
        for ex in d.values():
            sx.sx_executor_destroy(ex)
    sx.sx_executor_destroy(e)
    sx.sx_target_destroy(t)
    if dist:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--shard", action="store_true",
                    help="split each logical n-element array into one contiguous block per rank "
                         "(Section 4.1's block allocator; strong scaling) instead of one replica per rank")
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 27,
                    help="elements per array; the per-pass events include host launch time once a "
                         "kernel runs shorter than its launch (below ~2^22): use --sweep there")
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64", help="type of the timed STREAM passes")
    ap.add_argument("--q", type=float, default=Q, help="STREAM's scalar (Listing 4: 3.0)")
    ap.add_argument("--seed", type=int, default=None, help="base seed of the seeded inputs")
    ap.add_argument("--init", choices=["uniform", "closed-form"], default="uniform",
                    help="seeded uniform [-1,1) inputs, or a=1, b=2, c=0")
    ap.add_argument("--stream-doubling", action="store_true",
                    help="double a once after construction, as classic STREAM does before timing")
    ap.add_argument("--variant", choices=["auto", "vector", "bulk", "tma", "tma_tensor"], default="auto",
                    help="kernel family of the timed passes (auto: the tuner table)")
    ap.add_argument("--dram-mix", action="store_true",
                    help="instead of the step benchmark: the DRAM rate of stores only (fill), one read per "
                         "write (copy) and two reads per write (add) on FP64 arrays of --n elements")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the step benchmark: the size sweep, vector vs the two TMA bulk-copy families")
    ap.add_argument("--sweep-lo", type=int, default=10)
    ap.add_argument("--sweep-hi", type=int, default=29)
    ap.add_argument("--ref-n", type=int, default=1 << 22)
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--tune-cache", default="", help="extra tuner table to load and to save to")
    ap.add_argument("--tune-table", default=os.path.join(ROOT, "paper_2206_06302_b300", "tune_b300.json"),
                    help="tuner table loaded first (the one shipped for B300)")
    ap.add_argument("--retune", action="store_true", help="tune every pass kernel again")
    ap.add_argument("--tune-n", type=int, default=0,
                    help="size whose tuned launch shapes the pass kernels use (default: --n)")
    ap.add_argument("--quick", action="store_true", help="FP64 pass only (no FP32, e2e, sections)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=1 << 24)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--sections", default="batched,served,small,overlap,copies")
    ap.add_argument("--cpu-threads-n", type=int, default=1 << 25,
                    help="sample size of the threaded CPU baseline (0: skip)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-reps", type=int, default=10)
    ap.add_argument("--serve-count", type=int, default=2000)
    ap.add_argument("--serve-loads", default="0.5,0.8,0.95")
    ap.add_argument("--serve-load-reps", type=int, default=3, help="replays per offered load and mode")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.dram_mix:
        return run_dram_mix(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
