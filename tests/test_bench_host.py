"""Host logic of bench.py, on CPU: the reconstruction count inside the timed passes, the compact
batched and served comparisons that close the JSON line, and the served workload's byte
accounting (STREAM bytes against the DRAM bytes of each serving mode)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reseeds_between():
    assert bench.reseeds_between(5, 20) == 0
    assert bench.reseeds_between(0, 100) == 0 and bench.reseeds_between(0, 101) == 1
    assert bench.reseeds_between(95, 10) == 1 and bench.reseeds_between(5, 1000) == 10


def test_served_summary():
    runs = [dict(mode=m, offered_load=ld, p50_ms=p50, p99_ms=p99, **{"GB/s": g})
            for m, ld, p50, p99, g in (("continuous", 0.5, 0.1, 1.0, 10.0), ("fifo", 0.5, 0.2, 2.0, 10.0),
                                        ("continuous", 0.9, 0.1, 3.0, 18.0), ("fifo", 0.9, 5.0, 2.5, 17.0))]
    s = bench.served_summary({"runs": runs, "saturation_GB/s": {"continuous": 8.0, "fifo": 5.0}})
    assert s["saturation_gain"] == 1.6 and s["beats_fifo"]["throughput"]
    assert s["loads"]["0.5"]["p99_ms"] == [1.0, 2.0] and s["loads"]["0.9"]["GB/s"] == [18.0, 17.0]
    assert not s["beats_fifo"]["p99_every_load"]  # 3.0 > 2.5 at 0.9


def test_served_summary_takes_the_median_replay():
    """Three replays per load and mode: the summary reports the median of each figure, with every
    replay's p99 beside it, so that one replay's outlier does not decide the comparison."""
    runs = [dict(mode=m, offered_load=0.5, replay=r, p50_ms=p50, p99_ms=p99, **{"GB/s": 10.0})
            for m, r, p50, p99 in (("continuous", 0, 0.1, 1.1), ("fifo", 0, 0.2, 2.1),
                                   ("continuous", 1, 0.3, 2.9), ("fifo", 1, 0.2, 2.0),
                                   ("continuous", 2, 0.1, 1.2), ("fifo", 2, 0.25, 2.2))]
    s = bench.served_summary({"runs": runs, "saturation_GB/s": {"continuous": 8.0, "fifo": 5.0}})
    ld = s["loads"]["0.5"]
    assert ld["p99_ms"] == [1.2, 2.1] and ld["p50_ms"] == [0.1, 0.2]
    assert ld["p99_runs_ms"] == [[1.1, 2.9, 1.2], [2.1, 2.0, 2.2]]
    assert s["beats_fifo"]["p99_every_load"]


def test_batched_summary():
    b = {"workload": "w", "graph_ms": 1.0, "percall_ms": 2.0, "graph_GB/s": 10.0, "percall_GB/s": 5.0,
         "percall_graph_ms": 1.5, "percall_graph_GB/s": 6.7, "speedup_vs_percall_graph": 1.5,
         "speedup": 2.0, "completion_ms_p50": {"graph": 0.5, "percall": 1.0},
         "completion_ms_p99": {"graph": 0.9, "percall": 1.9}, "graph_equals_percall_8_instances": True,
         "noalloc": {"device_ms": 1.1, "host_us_per_call_median": 900.0, "graph_launch_host_us_median": 2.0}}
    s = bench.batched_summary(b)
    assert s["beats_percall"] == {"throughput": True, "throughput_vs_percall_graph": True, "p99": True}
    assert s["noalloc_host_us_per_call"] == 900.0 and s["ms"]["percall_graph"] == 1.5


def test_served_workload_byte_accounting():
    import paper_2206_06302_b300 as sx
    dram = {}
    reqs, work, nbytes = bench.served_workload(sx, 99, 300, dram)
    assert len(work) == len(nbytes) == 300
    # the per-call FIFO moves every STREAM byte through DRAM; construct-then-operate pieces only
    # store (x, y, out): 3 of 5 arrays for add/triad, 2 of 3 for copy/scale
    assert dram["fifo"] == sum(nbytes)
    written = sum(r["n"] * (8 if r["dtype"] == "f64" else 4) * (3 if r["op"] in ("add", "triad") else 2)
                  for r in reqs)
    assert dram["continuous"] == written < dram["fifo"]


def test_shard_requests_deal_every_request_once():
    import stream_inputs as si
    reqs = si.poisson_requests(5, 1001, rate_per_s=1.0)
    for world in (1, 2, 3, 8):
        parts = [bench.shard_requests(reqs, world, r) for r in range(world)]
        assert sum(len(p) for p in parts) == len(reqs)
        seen = sorted((r["t"], r["seed"]) for p in parts for r in p)
        assert seen == sorted((r["t"], r["seed"]) for r in reqs)
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    import paper_2206_06302_b300 as sx
    full = bench.served_workload(sx, 5, 1001)[2]
    halves = [bench.served_workload(sx, 5, 1001, None, 2, r)[2] for r in (0, 1)]
    assert sorted(full) == sorted(halves[0] + halves[1])


def test_batched_instances_assigned_whole_in_blocks():
    """--shard gives each rank a contiguous block of the one batched workload (sx_block_partition
    over the instance count): the blocks put together are the whole list, in order."""
    import paper_2206_06302_b300 as sx
    import stream_inputs as si
    inst = si.batched_instances(si.BASE_SEED, 4096)
    for world in (1, 2, 3, 8):
        parts = []
        for r in range(world):
            first, count = bench.shard_block(sx, len(inst), world, r)
            parts.extend(inst[first:first + count])
        assert parts == inst


def test_clock_summary_takes_the_timed_window():
    """NVML samples: only those inside the timed region count; reason bits are named (the idle
    bit is not a throttle reason); with no window, every sample counts."""
    samples = [(0.0, 1000, 0x1), (1.0, 2032, 0x0), (1.1, 2032, 0x4), (1.2, 1990, 0x0), (5.0, 800, 0x8)]
    s = bench.clock_summary(samples, (0.9, 1.3), 2032)
    assert s["sm_mhz"] == 2032 and s["samples"] == 3 and s["reasons"] == ["sw_power_cap"]
    s = bench.clock_summary(samples, (None, None), 2032)
    assert s["samples"] == 5 and s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.clock_summary([], (0, 1), 2032) is None
