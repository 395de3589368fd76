"""GPU tests of sx_batch_run_noalloc, the batch launch that allocates no device memory.

That call exists for callers that must not allocate: a process whose device memory already
belongs to another allocator (a framework's caching pool that has reserved the free memory),
or a latency-bound loop that cannot afford cudaMalloc/cudaFree, which may synchronize the whole
device.  Its tables live in a static device array shared by every call.  These tests check, bit
for bit as every other GPU test here:

* every instance's output against the oracle (SEED items against the seeded generator), on two
  calls in a row, with instances off the vector alignment, and against the ordinary entry point
  (sx_batch_create + sx_batch_launch);
* two different item sets enqueued back to back on one stream with no synchronization between
  the calls (the second call's table copy must wait, in stream order, for the first kernel);
* that a stream under CUDA-graph capture is refused, and sizes beyond the static array too,
  before anything runs.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
import paper_2206_06302_b300 as sx
import stream_inputs as si
from gpu_util import assert_bitwise

pytestmark = pytest.mark.gpu

OPS = [sx.SX_OP_COPY, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_TRIAD, sx.SX_OP_SEED]
OPN = {sx.SX_OP_COPY: "copy", sx.SX_OP_SCALE: "scale", sx.SX_OP_ADD: "add", sx.SX_OP_TRIAD: "triad"}


class Workload:
    """`count` instances of every op and both types carved from one device buffer, inputs
    seeded, every third instance off the vector alignment by whole elements."""

    def __init__(self, count, seed, hi_exp=16):
        import torch
        lens = si.log_uniform_lengths(si.word_scalar(seed, 1), count, 0, hi_exp)
        self.specs, total = [], 0
        for k in range(count):
            es = 8 if k % 2 == 0 else 4
            off = (k % 4) * es if k % 3 == 0 else 0
            regions = []
            for _ in range(3):
                total = (total + 255) // 256 * 256 + off
                regions.append(total)
                total += int(lens[k]) * es
            op = OPS[k % len(OPS)]
            self.specs.append(dict(op=op, dt=np.float64 if es == 8 else np.float32, n=int(lens[k]),
                                   regions=regions, q=-1.0 if op == sx.SX_OP_SEED else [3.0, -0.3, 0.5][k % 3],
                                   seed=si.word_scalar(seed, 500 + k), base=k))
        self.buf = torch.zeros(total + 256, dtype=torch.uint8, device="cuda")
        self.base = self.buf.data_ptr()
        self.inputs = []
        for k, s in enumerate(self.specs):
            x, y = (si.uniform(si.array_seed(seed, j, k), s["n"], s["dt"]) for j in (0, 1))
            self.inputs.append((x, y))
            for arr, r in ((x, s["regions"][0]), (y, s["regions"][1])):
                self.buf[r:r + arr.nbytes] = torch.from_numpy(arr.view(np.uint8)).cuda()
        torch.cuda.synchronize()

    def items(self):
        return [sx.sx_batch_item(op=s["op"], dtype=sx.SX_F64 if s["dt"] == np.float64 else sx.SX_F32, n=s["n"],
                                 x=self.base + s["regions"][0], y=self.base + s["regions"][1],
                                 out=self.base + s["regions"][2], q=s["q"], q2=1.0, seed=s["seed"],
                                 index_base=s["base"]) for s in self.specs]

    def clear_outputs(self):
        import torch
        for s in self.specs:
            r = s["regions"][2]
            self.buf[r:r + s["n"] * np.dtype(s["dt"]).itemsize] = 0xEE
        torch.cuda.synchronize()

    def outputs(self):
        import torch
        torch.cuda.synchronize()
        h = self.buf.cpu().numpy()
        return [h[s["regions"][2]:s["regions"][2] + s["n"] * np.dtype(s["dt"]).itemsize].view(s["dt"]).copy()
                for s in self.specs]

    def check_oracle(self, what):
        """Every instance against the oracle (SEED: the seeded generator at its index base)."""
        for k, (got, s) in enumerate(zip(self.outputs(), self.specs)):
            x, y = self.inputs[k]
            if s["op"] == sx.SX_OP_SEED:
                want = si.uniform(s["seed"], s["n"], s["dt"], -1.0, 1.0, start=s["base"])
            else:
                want = oracle.apply(OPN[s["op"]], x, y, s["q"])
            assert_bitwise(got, want, f"{what}: instance {k} (op {s['op']}, {s['dt'].__name__}, n={s['n']})")


def test_noalloc_matches_the_oracle_and_the_batch_entry_point(target):
    w = Workload(300, seed=77)
    stream = sx.sx_target_stream(target)
    # the ordinary entry point (its tables in memory it allocates)
    b = sx.sx_batch_create(target, w.items())
    w.clear_outputs()
    sx.sx_batch_launch(b)
    sx.sx_target_synchronize(target)
    want = w.outputs()
    sx.sx_batch_destroy(b)
    for call in range(2):  # two calls in a row reuse the static tables
        w.clear_outputs()
        sx.sx_batch_run_noalloc(stream, w.items())
        sx.sx_target_synchronize(target)
        w.check_oracle(f"call {call}")
        for k, (g, ref) in enumerate(zip(w.outputs(), want)):
            assert_bitwise(g, ref, f"call {call}: instance {k} against sx_batch_launch")
    # another launch shape, still the oracle's bits
    w.clear_outputs()
    sx.sx_batch_run_noalloc(stream, w.items(), dict(chunk_bytes=16384, threads=128, blocks_per_sm=2,
                                                   vec_bytes=16))
    sx.sx_target_synchronize(target)
    w.check_oracle("small tiles")


def test_noalloc_back_to_back_on_one_stream(target):
    """Two different item sets, enqueued one after the other on one stream with no
    synchronization between the calls: the second call's tables overwrite the first's in the
    shared array only after the first kernel has run (stream order), so both sets come out as
    the oracle's.  The sets use different launch shapes, so their tile tables differ too."""
    a = Workload(257, seed=91, hi_exp=18)
    b = Workload(101, seed=92, hi_exp=14)
    stream = sx.sx_target_stream(target)
    for rep in range(2):
        a.clear_outputs()
        b.clear_outputs()
        sx.sx_batch_run_noalloc(stream, a.items(), dict(chunk_bytes=16384, threads=256, blocks_per_sm=2,
                                                       vec_bytes=32))
        sx.sx_batch_run_noalloc(stream, b.items())
        sx.sx_batch_run_noalloc(stream, a.items(), dict(chunk_bytes=65536, threads=512, blocks_per_sm=1,
                                                       vec_bytes=16))
        sx.sx_target_synchronize(target)
        a.check_oracle(f"rep {rep}: first set")
        b.check_oracle(f"rep {rep}: second set")


def test_noalloc_refused_while_the_stream_is_captured(target):
    """Under CUDA-graph capture the call returns SX_ERR_STATE and enqueues nothing; the same
    call then runs once the capture has ended."""
    import torch
    w = Workload(20, seed=93)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    marker = torch.zeros(1, device="cuda")
    with torch.cuda.graph(g, stream=s):
        marker.add_(1.0)  # the graph has a node of its own
        with pytest.raises(sx.SxError) as ei:
            sx.sx_batch_run_noalloc(s.cuda_stream, w.items())
    assert ei.value.status == sx.SX_ERR_STATE and "captured" in str(ei.value)
    w.clear_outputs()
    sx.sx_batch_run_noalloc(s.cuda_stream, w.items())
    s.synchronize()
    w.check_oracle("after the capture")
    del g


def test_noalloc_refuses_sizes_beyond_its_array(target):
    w = Workload(4, seed=78)
    items = w.items()
    too_many = [items[0]] * (sx.SX_NOALLOC_MAX_ITEMS + 1)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_batch_run_noalloc(sx.sx_target_stream(target), too_many)
    assert ei.value.status == sx.SX_ERR_INVALID and "static scratch" in str(ei.value)
    # one long item cut into more tiles than the tile table holds
    big = sx.sx_batch_item(op=sx.SX_OP_COPY, dtype=sx.SX_F64, n=(sx.SX_NOALLOC_MAX_TILES + 1) * 1024,
                           x=items[0].x, y=items[0].y, out=items[0].out, q=0.0)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_batch_run_noalloc(sx.sx_target_stream(target), [big], dict(chunk_bytes=16384))
    assert ei.value.status == sx.SX_ERR_INVALID and "work tiles" in str(ei.value)
    sx.sx_batch_run_noalloc(sx.sx_target_stream(target), [])  # an empty batch is a no-op
