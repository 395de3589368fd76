"""GPU test of sx_batch_run_noalloc, the batch launch that allocates no device memory.

That call exists for callers that must not allocate: a process whose device memory already
belongs to another allocator (a framework's caching pool that has reserved the free memory),
or a latency-bound loop that cannot afford cudaMalloc/cudaFree, which may synchronize the whole
device.  Its tables live in a static device array shared by every call.  This test checks that
two calls in a row on the same inputs give exactly the outputs of the ordinary entry point
(sx_batch_create + sx_batch_launch), bit for bit as every other GPU test here, and that sizes
beyond the static array are refused before anything runs.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import paper_2206_06302_b300 as sx
import stream_inputs as si

pytestmark = pytest.mark.gpu

OPS = [sx.SX_OP_COPY, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_TRIAD, sx.SX_OP_SEED]


def _workload(count, seed):
    """`count` instances of every op and both types carved from one device buffer, inputs
    seeded, every third instance off the vector alignment.  Returns (buffer, items, outputs)."""
    import torch
    lens = si.log_uniform_lengths(si.word_scalar(seed, 1), count, 0, 16)
    specs, total = [], 0
    for k in range(count):
        es = 8 if k % 2 == 0 else 4
        off = (k % 4) * es if k % 3 == 0 else 0
        regions = []
        for _ in range(3):
            total = (total + 255) // 256 * 256 + off
            regions.append(total)
            total += int(lens[k]) * es
        specs.append((OPS[k % len(OPS)], es, int(lens[k]), regions))
    buf = torch.zeros(total + 256, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    items, outs = [], []
    for k, (op, es, n, r) in enumerate(specs):
        dt = np.float64 if es == 8 else np.float32
        for j in (0, 1):
            v = si.uniform(si.array_seed(seed, j, k), n, dt)
            buf[r[j]:r[j] + n * es] = torch.from_numpy(v.view(np.uint8)).cuda()
        items.append(sx.sx_batch_item(
            op=op, dtype=sx.SX_F64 if es == 8 else sx.SX_F32, n=n, x=base + r[0], y=base + r[1],
            out=base + r[2], q=-1.0 if op == sx.SX_OP_SEED else [3.0, -0.3, 0.5][k % 3],
            q2=1.0, seed=si.word_scalar(seed, 500 + k), index_base=k))
        outs.append((r[2], n * es))
    torch.cuda.synchronize()
    return buf, items, outs


def _outputs(buf, outs):
    import torch
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    return [h[o:o + nb].copy() for o, nb in outs]


def _clear(buf, outs):
    import torch
    for o, nb in outs:
        buf[o:o + nb] = 0xEE
    torch.cuda.synchronize()


def test_noalloc_matches_the_batch_entry_point(target):
    buf, items, outs = _workload(300, seed=77)
    stream = sx.sx_target_stream(target)
    # the ordinary entry point (its tables in memory it allocates) gives the reference outputs
    b = sx.sx_batch_create(target, items)
    sx.sx_batch_launch(b)
    sx.sx_target_synchronize(target)
    want = _outputs(buf, outs)
    sx.sx_batch_destroy(b)
    for call in range(2):  # two calls in a row reuse the static tables
        _clear(buf, outs)
        sx.sx_batch_run_noalloc(stream, items)
        sx.sx_target_synchronize(target)
        got = _outputs(buf, outs)
        for k, (g, w) in enumerate(zip(got, want)):
            assert np.array_equal(g, w), f"call {call}: instance {k} differs"
    # another launch shape, still the same bits
    _clear(buf, outs)
    sx.sx_batch_run_noalloc(stream, items, dict(chunk_bytes=16384, threads=128, blocks_per_sm=2,
                                                vec_bytes=16))
    sx.sx_target_synchronize(target)
    for k, (g, w) in enumerate(zip(_outputs(buf, outs), want)):
        assert np.array_equal(g, w), f"small tiles: instance {k} differs"


def test_noalloc_refuses_sizes_beyond_its_array(target):
    buf, items, outs = _workload(4, seed=78)
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
