"""GPU parity of the STREAM kernels against the CPU oracle, through the C ABI.

Bar: bit-for-bit equality (binary64 and binary32) on seeded inputs, for every kernel family and
launch shape, at sizes that span several tiles with ragged heads and tails, misaligned and
aliased operands, the hand-derived rounding cases, and STREAM's closed form.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2206_06302_b300 as sx
import stream_inputs as si
from gpu_util import CODE, assert_bitwise, bits, empty, to_device, to_host
from test_oracle_pins import rounding_cases

pytestmark = pytest.mark.gpu

OPS = {"copy": sx.SX_OP_COPY, "scale": sx.SX_OP_SCALE, "add": sx.SX_OP_ADD,
       "triad": sx.SX_OP_TRIAD}
SIZES = [1, 2, 3, 5, 7, 8, 31, 33, 255, 257, 1000, 4099, 65537, (1 << 20) + 3]

CFGS = [
    None,  # executor default / tuner table
    dict(variant=sx.SX_VARIANT_VECTOR, threads=256, vec_bytes=16, unroll=1),
    dict(variant=sx.SX_VARIANT_VECTOR, threads=128, vec_bytes=32, unroll=4, blocks_per_sm=2,
         fp64_mul=1),
    dict(variant=sx.SX_VARIANT_VECTOR, threads=1024, vec_bytes=32, unroll=2, cache_hint=1,
         fp64_mul=2),
    dict(variant=sx.SX_VARIANT_VECTOR, threads=512, vec_bytes=16, unroll=4, blocks_per_sm=1,
         cache_hint=1, fp64_mul=1),
    # TMA bulk-copy staging: tiles of 1 KiB make even the mid sizes span many tiles and blocks
    dict(variant=sx.SX_VARIANT_BULK, threads=128, blocks_per_sm=1, tile_bytes=1024, stages=2),
    dict(variant=sx.SX_VARIANT_BULK, threads=256, blocks_per_sm=2, tile_bytes=4096, stages=4,
         fp64_mul=1),
    dict(variant=sx.SX_VARIANT_BULK, threads=512, blocks_per_sm=1, tile_bytes=16384, stages=6,
         fp64_mul=2),
    dict(variant=sx.SX_VARIANT_BULK, threads=256, blocks_per_sm=1, tile_bytes=32768, stages=3),
    # TMA both ways (results computed in place in shared memory and written by bulk stores)
    dict(variant=sx.SX_VARIANT_TMA, threads=96, blocks_per_sm=1, tile_bytes=1024, stages=2),
    dict(variant=sx.SX_VARIANT_TMA, threads=128, blocks_per_sm=2, tile_bytes=4096, stages=3,
         fp64_mul=1),
    dict(variant=sx.SX_VARIANT_TMA, threads=512, blocks_per_sm=1, tile_bytes=16384, stages=6,
         fp64_mul=2),
    dict(variant=sx.SX_VARIANT_TMA, threads=256, blocks_per_sm=4, tile_bytes=8192, stages=4),
    # the same with 2-D tensor-map copies (rows of 256 elements; boxes of 1..16 rows)
    dict(variant=sx.SX_VARIANT_TMA_TENSOR, threads=96, blocks_per_sm=1, tile_bytes=2048, stages=2),
    dict(variant=sx.SX_VARIANT_TMA_TENSOR, threads=128, blocks_per_sm=2, tile_bytes=4096, stages=3,
         fp64_mul=1),
    dict(variant=sx.SX_VARIANT_TMA_TENSOR, threads=256, blocks_per_sm=1, tile_bytes=16384, stages=4,
         fp64_mul=2),
    # each family's default shape (zero fields: the per-kernel shapes measured fastest at 2^27)
    dict(variant=sx.SX_VARIANT_BULK, fp64_mul=2),
    dict(variant=sx.SX_VARIANT_TMA, fp64_mul=2),
    dict(variant=sx.SX_VARIANT_TMA_TENSOR, fp64_mul=2),
]


def _inputs(n, dt, salt=0):
    x = si.uniform(si.array_seed(1000 + salt, 0, n), n, dt)
    y = si.uniform(si.array_seed(1000 + salt, 1, n), n, dt)
    return x, y


def _run_op(target, cfg, op, x, y, q, dt):
    e = sx.sx_executor_create(target, sx.SX_PAR, cfg)
    try:
        dx, dy, do = to_device(target, x), to_device(target, y), empty(target, dt, x.size)
        try:
            sx.sx_execute(e, OPS[op], dx, dy, do, q)
            got = to_host(do)
            assert sx.sx_array_guard_ok(do), "write past the end of the output"
        finally:
            for a in (dx, dy, do):
                sx.sx_free(a)
    finally:
        sx.sx_executor_destroy(e)
    return got


@pytest.mark.parametrize("cfg", range(len(CFGS)))
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("op", list(OPS))
def test_parity_sizes(target, op, dt, cfg):
    for n in SIZES:
        x, y = _inputs(n, dt)
        for q in (3.0, -0.1):
            got = _run_op(target, CFGS[cfg], op, x, y, q, dt)
            assert_bitwise(got, oracle.apply(op, x, y, q), f"{op} {dt.__name__} n={n} q={q}")


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_empty_arrays_are_noops(target, executor, dt):
    a, b = empty(target, dt, 0), empty(target, dt, 0)
    for op in OPS:
        sx.sx_execute(executor, OPS[op], a, a, b, 3.0)
    sx.sx_free(a)
    sx.sx_free(b)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("op", list(OPS))
def test_misaligned_and_mixed_offsets(target, executor, op, dt):
    """Borrowed arrays at element offsets: equal offsets take the vector path with scalar head
    and tail; unequal offsets (modulo the vector width) take the element path."""
    import torch
    n = 70001
    es = np.dtype(dt).itemsize
    tdt = torch.float64 if dt == np.float64 else torch.float32
    x, y = _inputs(n, dt, 7)
    want = oracle.apply(op, x, y, 3.0)
    for ox, oy, oo in [(1, 1, 1), (3, 3, 3), (0, 1, 2), (5, 0, 5), (2, 2, 0)]:
        bx = torch.zeros(n + 8, dtype=tdt, device="cuda")
        by = torch.zeros(n + 8, dtype=tdt, device="cuda")
        bo = torch.full((n + 8,), -7.0, dtype=tdt, device="cuda")
        bx[ox:ox + n] = torch.from_numpy(x).cuda()
        by[oy:oy + n] = torch.from_numpy(y).cuda()
        torch.cuda.synchronize()
        ax = sx.sx_array_wrap(target, sx.SX_F64 if es == 8 else sx.SX_F32, bx.data_ptr() + ox * es, n)
        ay = sx.sx_array_wrap(target, sx.SX_F64 if es == 8 else sx.SX_F32, by.data_ptr() + oy * es, n)
        ao = sx.sx_array_wrap(target, sx.SX_F64 if es == 8 else sx.SX_F32, bo.data_ptr() + oo * es, n)
        sx.sx_execute(executor, OPS[op], ax, ay, ao, 3.0)
        out = bo.cpu().numpy()
        assert_bitwise(out[oo:oo + n], want, f"{op} offsets {(ox, oy, oo)}")
        assert np.all(out[:oo] == -7.0) and np.all(out[oo + n:] == -7.0), "wrote outside the range"
        for a in (ax, ay, ao):
            sx.sx_free(a)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("op", list(OPS))
def test_output_aliases_input(target, executor, op, dt):
    n = 100003
    x, y = _inputs(n, dt, 3)
    want = oracle.apply(op, x, y, 3.0)
    dx, dy = to_device(target, x), to_device(target, y)
    sx.sx_execute(executor, OPS[op], dx, dy, dx, 3.0)  # out = x
    assert_bitwise(to_host(dx), want, f"{op} out=x")
    if op in ("add", "triad"):
        dx2 = to_device(target, x)
        sx.sx_execute(executor, OPS[op], dx2, dy, dy, 3.0)  # out = y
        assert_bitwise(to_host(dy), want, f"{op} out=y")
        sx.sx_free(dx2)
    sx.sx_free(dx)
    sx.sx_free(dy)


def test_argument_errors(target, executor):
    import torch
    a = empty(target, np.float64, 100)
    b = empty(target, np.float64, 101)
    c = empty(target, np.float32, 100)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_copy(executor, a, b)
    assert ei.value.status == sx.SX_ERR_INVALID
    with pytest.raises(sx.SxError) as ei:
        sx.sx_copy(executor, a, c)
    assert ei.value.status == sx.SX_ERR_DTYPE
    buf = torch.zeros(200, dtype=torch.float64, device="cuda")
    p1 = sx.sx_array_wrap(target, sx.SX_F64, buf.data_ptr(), 100)
    p2 = sx.sx_array_wrap(target, sx.SX_F64, buf.data_ptr() + 8 * 50, 100)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_copy(executor, p1, p2)
    assert ei.value.status == sx.SX_ERR_OVERLAP
    with pytest.raises(sx.SxError) as ei:
        sx.sx_executor_create(target, sx.SX_PAR, dict(variant=sx.SX_VARIANT_VECTOR, threads=100))
    assert ei.value.status == sx.SX_ERR_INVALID
    u = empty(target, np.uint8, 100)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_copy(executor, u, u)
    assert ei.value.status == sx.SX_ERR_DTYPE
    for h in (a, b, c, p1, p2, u):
        sx.sx_free(h)


@pytest.mark.parametrize("variant", [sx.SX_VARIANT_BULK, sx.SX_VARIANT_TMA, sx.SX_VARIANT_TMA_TENSOR])
def test_staging_shape_for_one_input_only(target, variant):
    """A staging shape of 3 x 64 KiB fits shared memory for one input array but not for two: the
    executor takes it, copy and scale run with it (oracle bits), add and triad refuse it."""
    e = sx.sx_executor_create(target, sx.SX_PAR, dict(variant=variant, threads=256, blocks_per_sm=1,
                                                      tile_bytes=65536, stages=3))
    n = (1 << 20) + 3
    x, y = _inputs(n, np.float64, salt=5)
    dx, dy, do = to_device(target, x), to_device(target, y), empty(target, np.float64, n)
    sx.sx_copy(e, dx, do)
    assert_bitwise(to_host(do), oracle.copy(x), "copy")
    sx.sx_transform_scale(e, dx, do, 3.0)
    assert_bitwise(to_host(do), oracle.scale(x, 3.0), "scale")
    for op in (sx.SX_OP_ADD, sx.SX_OP_TRIAD):
        with pytest.raises(sx.SxError) as ei:
            sx.sx_execute(e, op, dx, dy, do, 3.0)
        assert ei.value.status == sx.SX_ERR_INVALID
    for h in (dx, dy, do):
        sx.sx_free(h)
    sx.sx_executor_destroy(e)


def test_tensor_map_tiles_are_whole_rows(target):
    """TMA_TENSOR tiles are boxes of whole 256-element rows: a tile of 3 KiB is refused, and an
    array shorter than one row (all of it done element by element) gives the oracle's bits."""
    with pytest.raises(sx.SxError) as ei:
        sx.sx_executor_create(target, sx.SX_PAR, dict(variant=sx.SX_VARIANT_TMA_TENSOR, threads=128,
                                                      blocks_per_sm=1, tile_bytes=3072, stages=2))
    assert ei.value.status == sx.SX_ERR_INVALID
    e = sx.sx_executor_create(target, sx.SX_PAR, dict(variant=sx.SX_VARIANT_TMA_TENSOR, threads=128,
                                                      blocks_per_sm=1, tile_bytes=2048, stages=2))
    for n in (255, 256, 511, 513):
        x, y = _inputs(n, np.float64, salt=n)
        dx, dy, do = to_device(target, x), to_device(target, y), empty(target, np.float64, n)
        sx.sx_transform_triad(e, dx, dy, do, 3.0)
        assert_bitwise(to_host(do), oracle.triad(x, y, 3.0), f"n={n}")
        assert sx.sx_array_guard_ok(do)
        for h in (dx, dy, do):
            sx.sx_free(h)
    sx.sx_executor_destroy(e)


def test_budget_is_enforced_on_the_host():
    t = sx.sx_target_create_ext(0, None, 1 << 20)
    a = sx.sx_alloc(t, sx.SX_F64, 1000)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_alloc(t, sx.SX_F64, 1 << 20)
    assert ei.value.status == sx.SX_ERR_OOM
    info = sx.sx_target_info_get(t)
    assert info["used"] == 8192 + 256 and info["budget"] == 1 << 20
    sx.sx_free(a)
    assert sx.sx_target_info_get(t)["used"] == 0
    sx.sx_target_destroy(t)


def test_rounding_cases_on_gpu(target, executor):
    for dt, op, x, y, q, exp, note in rounding_cases():
        n = 77
        xa = np.full(n, x, dt)
        ya = np.full(n, y if y is not None else 0, dt)
        dx, dy, do = to_device(target, xa), to_device(target, ya), empty(target, dt, n)
        sx.sx_execute(executor, OPS[op], dx, dy, do, q)
        assert_bitwise(to_host(do), np.full(n, exp, dt), f"{op} {note}")
        for a in (dx, dy, do):
            sx.sx_free(a)


def _stream_device(target, executor, a, b, c, q, iters, fused=False):
    da, db, dc = to_device(target, a), to_device(target, b), to_device(target, c)
    (sx.sx_stream_fused if fused else sx.sx_stream_iter)(executor, da, db, dc, q, iters)
    out = tuple(to_host(h) for h in (da, db, dc))
    for h in (da, db, dc):
        sx.sx_free(h)
    return out


@pytest.mark.parametrize("fused", [False, True])
def test_closed_form_fp64_k10_config(target, executor, fused):
    """STREAM FP64, n=2^20, a=1 b=2 c=0 q=3, 10 passes: the closed form, exactly."""
    n = 1 << 20
    a, b, c = si.closed_form_arrays(n, np.float64)
    ga, gb, gc = _stream_device(target, executor, a, b, c, 3.0, 10, fused)
    assert np.all(ga == 576650390625.0) and np.all(gb == 115330078125.0)
    assert np.all(gc == 153773437500.0)


@pytest.mark.parametrize("fused", [False, True])
def test_closed_form_fp32_k6(target, executor, fused):
    n = 12345
    a, b, c = si.closed_form_arrays(n, np.float32)
    ga, gb, gc = _stream_device(target, executor, a, b, c, 3.0, 6, fused)
    assert np.all(ga == 15.0 ** 6) and np.all(gb == 3 * 15.0 ** 5) and np.all(gc == 4 * 15.0 ** 5)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_stream_passes_match_oracle(target, executor, dt, fused):
    n = 65536 * 3 + 17
    for iters in (1, 4, 40):
        a, b, c = si.stream_arrays(n, dt, base_seed=77)
        ga, gb, gc = _stream_device(target, executor, a, b, c, 3.0, iters, fused)
        oracle.stream(a, b, c, 3.0, iters)
        assert_bitwise(ga, a, f"a iters={iters}")
        assert_bitwise(gb, b, f"b iters={iters}")
        assert_bitwise(gc, c, f"c iters={iters}")


@pytest.mark.parametrize("cfg", range(len(CFGS)))
def test_stream_iter_graphs_match_oracle(target, cfg):
    """Passes replayed from captured CUDA graphs (37 = 16 + 16 + 5 passes, then the same call
    again from the executor's cache) give the oracle's bits for every launch shape, including the
    bulk-copy families, in both types."""
    e = sx.sx_executor_create(target, sx.SX_PAR, CFGS[cfg])
    try:
        for dt, n in ((np.float64, 65536 + 7), (np.float32, 4099)):
            a, b, c = si.stream_arrays(n, dt, base_seed=91)
            da, db, dc = to_device(target, a), to_device(target, b), to_device(target, c)
            for _ in range(2):
                sx.sx_stream_iter(e, da, db, dc, 3.0, 37)
                oracle.stream(a, b, c, 3.0, 37)
                for got, want, nm in ((da, a, "a"), (db, b, "b"), (dc, c, "c")):
                    assert_bitwise(to_host(got), want, f"{nm} {dt.__name__}")
            for h in (da, db, dc):
                sx.sx_free(h)
    finally:
        sx.sx_executor_destroy(e)


def test_stream_iter_graph_cache_eviction(target):
    """More array sets than the executor keeps graphs for, then the first set again."""
    e = sx.sx_executor_create(target, sx.SX_PAR_TASK)
    n = 3001
    host = [si.stream_arrays(n, np.float64, base_seed=300 + k) for k in range(11)]
    dev = [[to_device(target, h) for h in hs] for hs in host]
    for k in list(range(11)) + [0, 1]:
        sx.sx_stream_iter(e, *dev[k], 3.0, 3)
        oracle.stream(*host[k], 3.0, 3)
    sx.sx_executor_wait(e)
    for k in range(11):
        for got, want in zip(dev[k], host[k]):
            assert_bitwise(to_host(got), want, f"set {k}")
    for d in dev:
        for h in d:
            sx.sx_free(h)
    sx.sx_executor_destroy(e)


def test_stream_iter_inside_a_caller_capture():
    """While the target's stream is being captured by the caller (torch.cuda.graph), the passes
    are launched directly into that capture; replaying the caller's graph runs them."""
    import torch
    import paper_2206_06302_b300 as pkg
    s = torch.cuda.Stream()
    t = pkg.target_on_torch_stream(0, s)
    e = sx.sx_executor_create(t, sx.SX_PAR_TASK)
    n = 10007
    a, b, c = si.stream_arrays(n, np.float64, base_seed=12)
    da, db, dc = to_device(t, a), to_device(t, b), to_device(t, c)
    sx.sx_target_synchronize(t)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sx.sx_stream_iter(e, da, db, dc, 3.0, 3)
    for _ in range(2):
        g.replay()
        oracle.stream(a, b, c, 3.0, 3)
    torch.cuda.synchronize()
    for got, want in zip((da, db, dc), (a, b, c)):
        assert_bitwise(to_host(got), want, "captured by the caller")
    for h in (da, db, dc):
        sx.sx_free(h)
    sx.sx_executor_destroy(e)
    sx.sx_target_destroy(t)


def test_fused_equals_four_launches_unaligned(target, executor):
    import torch
    n = 50001
    for dt, tdt, code in ((np.float64, torch.float64, sx.SX_F64), (np.float32, torch.float32, sx.SX_F32)):
        a, b, c = si.stream_arrays(n, dt, base_seed=5)
        oracle.stream(a, b, c, 3.0, 3)
        buf = torch.from_numpy(np.concatenate([np.zeros(1, dt), si.stream_arrays(n, dt, base_seed=5)[0],
                                               np.zeros(2 * n + 3, dt)])).cuda()
        es = np.dtype(dt).itemsize
        ha = sx.sx_array_wrap(target, code, buf.data_ptr() + es, n)
        hb = sx.sx_array_wrap(target, code, buf.data_ptr() + es * (n + 1), n)
        hc = sx.sx_array_wrap(target, code, buf.data_ptr() + es * (2 * n + 2), n)
        sx.sx_stream_fused(executor, ha, hb, hc, 3.0, 3)
        h = buf.cpu().numpy()
        assert_bitwise(h[1:n + 1], a, "a")
        assert_bitwise(h[n + 1:2 * n + 1], b, "b")
        assert_bitwise(h[2 * n + 2:3 * n + 2], c, "c")
        for x in (ha, hb, hc):
            sx.sx_free(x)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_seeded_construction_matches_generator(target, dt):
    for n, seed, lo, hi in ((1, 0, -1.0, 1.0), (100003, 12345, -1.0, 1.0), (4097, 99, 0.25, 7.5),
                            (300, 2 ** 63 + 5, -3.0, 0.1)):
        d = empty(target, dt, n)
        sx.sx_seed_uniform(d, seed, lo, hi)
        assert_bitwise(to_host(d), si.uniform(seed, n, dt, lo, hi), f"seed {seed}")
        sx.sx_free(d)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_seeded_construction_misaligned(target, dt):
    """Arrays that start off the 32-byte store alignment: scalar head, vector body, scalar tail."""
    import torch
    es = np.dtype(dt).itemsize
    code = sx.SX_F64 if dt == np.float64 else sx.SX_F32
    buf = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    for off in range(0, 32, es):
        for n, lo, hi in ((1, -1.0, 1.0), (7, -1.0, 1.0), (70001, -1.0, 1.0), (4099, 0.5, 2.0)):
            buf.zero_()
            torch.cuda.synchronize()
            d = sx.sx_array_wrap(target, code, buf.data_ptr() + 64 + off, n)
            sx.sx_seed_uniform(d, 31 + off, lo, hi)
            sx.sx_target_synchronize(target)
            h = buf.cpu().numpy()
            got = h[64 + off:64 + off + n * es].view(dt)
            assert_bitwise(got, si.uniform(31 + off, n, dt, lo, hi), f"offset {off} n {n}")
            assert not h[:64 + off].any() and not h[64 + off + n * es:].any(), "wrote outside the array"
            sx.sx_free(d)


def _small_k_indices(seed, count):
    """Indices i < count whose word gives |k| < 2^32 for lo = -1, hi = 1 (k = (w >> 11) - 2^52,
    the value k 2^-52): the words whose leading bit lies in the low half of k."""
    w = si.words(seed, count)
    k = (w >> np.uint64(11)).astype(np.int64) - (1 << 52)
    return np.nonzero(np.abs(k) < (1 << 32))[0]


def test_seeded_general_range_on_both_units(target):
    """A general [lo, hi) in binary64 takes three of every four elements through an integer-unit form
    (u assembled from the word's bits, the product by mul_rn_int; a short-significand span takes
    its short path).  Words with M = w >> 11 below 2^32 (u < 2^-21, found by the host generator)
    put the leading bit in the low half; at every 8-byte offset each such word meets both forms.
    Spans: long and short significands, negative, huge and tiny (products near the subnormal and
    overflow ends defer to the FP64 pipe)."""
    import torch
    seed, count = 777, 1 << 23
    w = si.words(seed, count)
    hits = np.nonzero((w >> np.uint64(11)) < np.uint64(1 << 32))[0]
    assert hits.size >= 2, "no small word in range"
    n = int(hits[-1]) + 8
    buf = torch.zeros(8 * n + 64, dtype=torch.uint8, device="cuda")
    ranges = [(0.25, 7.5), (-3.0, 0.1), (1.0, 1.0 + 2.0 ** -40), (5.0, -2.0),
              (-1.0e300, 1.0e300), (0.0, 2.0 ** -1000), (-1.0, 0.5), (1.0e-310, 3.0e-310)]
    for off in (0, 8, 16, 24):
        for lo, hi in ranges:
            d = sx.sx_array_wrap(target, sx.SX_F64, buf.data_ptr() + off, n)
            sx.sx_seed_uniform(d, seed, lo, hi)
            got = to_host(d)
            want = si.uniform(seed, n, np.float64, lo, hi)
            assert_bitwise(got, want, f"[{lo}, {hi}) at offset {off}")
            sx.sx_free(d)


def test_seeded_pm1_small_magnitudes(target):
    """The lo = -1, hi = 1 binary64 construction has a separate path for |k| < 2^32 (about one
    word in 2^20): such words, found by the host generator, must come out exact through the
    grid-wide kernel and through batched tiles, at head, vector-body and tail positions."""
    import torch
    seed, count = 4242, 1 << 23
    hits = _small_k_indices(seed, count)
    assert hits.size >= 2, "no small-magnitude word in range"
    n = int(hits[-1]) + 1
    d = empty(target, np.float64, n)
    sx.sx_seed_uniform(d, seed, -1.0, 1.0)
    ref = si.uniform(seed, n, np.float64)
    assert np.all(np.abs(ref[hits]) < 2.0 ** -20)
    assert_bitwise(to_host(d), ref, "seed_uniform")
    sx.sx_free(d)
    # batched tiles: each hit at the start, inside and at the end of a small item, with the
    # output at every 8-byte offset of the 32-byte vector alignment
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    items, expect = [], []
    at = 0
    for h in hits[:4]:
        for off in (0, 8, 16, 24):
            for lead, m in ((0, 40), (17, 40), (39, 40), (3, 5)):
                at = (at + 255) // 256 * 256 + off
                items.append(sx.sx_batch_item(op=sx.SX_OP_SEED, dtype=sx.SX_F64, n=m,
                                              out=buf.data_ptr() + at, q=-1.0, q2=1.0, seed=seed,
                                              index_base=int(h) - lead))
                expect.append((at, si.uniform(seed, m, np.float64, start=int(h) - lead)))
                at += 8 * m
    for cfg in (None, dict(chunk_bytes=16384, threads=64, blocks_per_sm=1, vec_bytes=16)):
        buf.zero_()
        torch.cuda.synchronize()
        b = sx.sx_batch_create(target, items, cfg)
        sx.sx_batch_launch(b)
        sx.sx_target_synchronize(target)
        sx.sx_batch_destroy(b)
        h = buf.cpu().numpy()
        for k, (o, e) in enumerate(expect):
            assert_bitwise(h[o:o + 8 * e.size].view(np.float64), e, f"item {k}")


def test_bulk_construct_fill(target):
    for dt in (np.float64, np.float32, np.uint8):
        d = empty(target, dt, 1001)
        sx.sx_bulk_construct(d, 2.0)
        assert np.all(to_host(d) == 2)
        sx.sx_bulk_destroy(d)  # Listing 1's pair to bulk_construct; frees nothing
        assert sx.sx_array_data(d)[1] == 1001
        sx.sx_free(d)
    # the value converted to the element type once, every element its bits (32-byte vector stores
    # in the body, element stores at a misaligned head and a ragged tail), nothing written past
    # the end of the array or outside a borrowed view
    values = {np.float64: (-0.0, 5e-324, float("inf"), 1.0 / 3.0), np.float32: (-0.0, 1e-45, float("-inf"), 1.0 / 3.0),
              np.uint8: (0.0, 97.0, 255.0)}
    for dt, vals in values.items():
        es = np.dtype(dt).itemsize
        for n in (1, 3, 31, 33, 4099, (1 << 20) + 5):
            for v in vals:
                want = np.full(n, v, dt) if dt != np.uint8 else np.full(n, int(v), dt)
                d = empty(target, dt, n)
                sx.sx_bulk_construct(d, v)
                assert_bitwise(to_host(d), want, f"fill {dt.__name__} n={n} v={v}")
                assert sx.sx_array_guard_ok(d)
                sx.sx_free(d)
        # a view starting off the 32-byte boundary inside a larger array of sentinels
        n = 5000
        big = to_device(target, np.full(n + 64, 7, dt))
        base = sx.sx_array_data(big)[0]
        for off in (1, 3, 5):
            view = sx.sx_array_wrap(target, CODE[np.dtype(dt)], base + off * es, n)
            sx.sx_bulk_construct(view, 1.0)
            got = to_host(big)
            assert np.all(got[off:off + n] == 1) and np.all(got[:off] == 7) and np.all(got[off + n:] == 7), off
            sx.sx_bulk_construct(view, 7.0)
            sx.sx_free(view)
        sx.sx_free(big)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_bulk_destroy(None)
    assert ei.value.status == sx.SX_ERR_INVALID


def test_to_upper_listing3(target, executor):
    text = np.frombuffer(b"helloworld" + bytes(range(256)) * 41 + b"tail", np.uint8).copy()
    for off in (0, 1, 5):
        s = text[off:].copy()
        ds, do = to_device(target, s), empty(target, np.uint8, s.size)
        sx.sx_transform_u8(executor, sx.SX_FN_TO_UPPER, ds, do)
        assert_bitwise(to_host(do), oracle.to_upper(s), "to_upper")
        sx.sx_transform_u8(executor, sx.SX_FN_TO_LOWER, do, do)
        assert to_host(do).tobytes() == s.tobytes().upper().lower()
        sx.sx_free(ds)
        sx.sx_free(do)


def test_futures_async_execute(target):
    e = sx.sx_executor_create(target, sx.SX_PAR_TASK)
    n = 1 << 22
    x, y = _inputs(n, np.float64, 11)
    dx, dy, do = to_device(target, x), to_device(target, y), empty(target, np.float64, n)
    f = sx.sx_execute_async(e, sx.SX_OP_TRIAD, dx, dy, do, 3.0)
    sx.sx_future_wait(f, 10000)
    assert sx.sx_future_test(f)
    ms = sx.sx_future_elapsed_ms(f)
    assert 0.0 < ms < 1000.0
    sx.sx_future_destroy(f)
    assert_bitwise(to_host(do), oracle.triad(x, y, 3.0))
    # fire and forget, then wait on the executor
    sx.sx_execute_async(e, sx.SX_OP_COPY, dx, None, do, 0.0, future=False)
    sx.sx_executor_wait(e)
    assert_bitwise(to_host(do), x)
    for a in (dx, dy, do):
        sx.sx_free(a)
    sx.sx_executor_destroy(e)


def test_stream_host_end_to_end(target, executor):
    n = 300007
    for dt in (np.float64, np.float32):
        a, b, c = si.stream_arrays(n, dt, base_seed=21)
        ha, hb, hc = a.copy(), b.copy(), c.copy()
        da, db, dc = (empty(target, dt, n) for _ in range(3))
        sx.sx_stream_host(executor, ha.ctypes.data, hb.ctypes.data, hc.ctypes.data, da, db, dc, 3.0, 3)
        oracle.stream(a, b, c, 3.0, 3)
        assert_bitwise(ha, a)
        assert_bitwise(hb, b)
        assert_bitwise(hc, c)
        for h in (da, db, dc):
            sx.sx_free(h)


def test_stream_host_reads_only_a(target, executor):
    """A pass writes c and b before reading them, so sx_stream_host copies only a to the device:
    host b and c holding NaNs (and device b, c holding other values) give the oracle's results of
    the seeded arrays; with zero passes all three arrays make the round trip unchanged."""
    n = (3 << 20) + 77
    for dt in (np.float64, np.float32):
        a, b, c = si.stream_arrays(n, dt, base_seed=24)
        ha, hb, hc = a.copy(), np.full(n, np.nan, dt), np.full(n, np.nan, dt)
        da, db, dc = (empty(target, dt, n) for _ in range(3))
        sx.sx_bulk_construct(db, -5.0)
        sx.sx_bulk_construct(dc, 9.0)
        sx.sx_stream_host(executor, ha.ctypes.data, hb.ctypes.data, hc.ctypes.data, da, db, dc, 3.0, 2)
        oracle.stream(a, b, c, 3.0, 2)
        for h, w, name in ((ha, a, "a"), (hb, b, "b"), (hc, c, "c")):
            assert_bitwise(h, w, f"{dt.__name__} {name}")
        x, y, z = si.stream_arrays(n, dt, base_seed=25)
        hx, hy, hz = x.copy(), y.copy(), z.copy()
        sx.sx_stream_host(executor, hx.ctypes.data, hy.ctypes.data, hz.ctypes.data, da, db, dc, 3.0, 0)
        for h, w, name in ((hx, x, "a"), (hy, y, "b"), (hz, z, "c")):
            assert_bitwise(h, w, f"{dt.__name__} round trip {name}")
        for d, w in ((da, x), (db, y), (dc, z)):
            assert_bitwise(to_host(d), w, "device copy after the round trip")
        for h in (da, db, dc):
            sx.sx_free(h)


def _random_doubles(n, seed):
    """Bit patterns spread over every binary64 exponent (zeros, subnormals, normals near the
    overflow threshold, infinities and NaNs included)."""
    w = si.words(seed, n)
    return w.view(np.float64).copy()


@pytest.mark.parametrize("variant", [sx.SX_VARIANT_VECTOR, sx.SX_VARIANT_BULK, sx.SX_VARIANT_TMA,
                                     sx.SX_VARIANT_TMA_TENSOR])
def test_integer_unit_product_is_bit_identical(target, executor, variant):
    """fp64_mul=1/2 (integer-unit RN-even product with FP64-pipe fallback) == fp64_mul=0 bit for
    bit on every bit pattern, and == the oracle wherever the result is not a generated NaN."""
    n = (1 << 20) + 5
    x = _random_doubles(n, 31)
    y = _random_doubles(n, 32)
    base = dict(variant=variant, threads=256)
    if variant in (sx.SX_VARIANT_BULK, sx.SX_VARIANT_TMA, sx.SX_VARIANT_TMA_TENSOR):
        base.update(tile_bytes=8192, stages=3, blocks_per_sm=1)
    else:
        base.update(vec_bytes=32, unroll=2)
    qs = [3.0, -0.1, 1.0, 2.0 ** -1022, 5e-324, 1.7976931348623157e308, 1e-300, 1e300,
          float.fromhex("0x1.fffffffffffffp-1"), -7.5, float("inf"), 0.0]
    for op in ("scale", "triad"):
        for q in qs:
            outs = [_run_op(target, dict(base, fp64_mul=mm), op, x, y, q, np.float64)
                    for mm in (0, 1, 2)]
            assert_bitwise(outs[1], outs[0], f"{op} q={q} mm=1")
            assert_bitwise(outs[2], outs[0], f"{op} q={q} mm=2")
            want = oracle.apply(op, x, y, q)
            ok = ~np.isnan(want)
            assert_bitwise(outs[1][ok], want[ok], f"{op} q={q} vs oracle")
            assert np.array_equal(np.isnan(outs[1]), np.isnan(want))


def test_integer_unit_product_near_thresholds(target, executor):
    """Products that round up into the next binade, to DBL_MAX / overflow, and across the
    normal/subnormal boundary."""
    vals = []
    for e in (-1022, -1021, -1000, -520, -1, 0, 1, 511, 1000, 1022, 1023):
        for m in ("0x1.0000000000000", "0x1.0000000000001", "0x1.fffffffffffff", "0x1.5555555555555",
                  "0x1.aaaaaaaaaaaab", "0x1.8000000000000", "0x1.7ffffffffffff"):
            v = float.fromhex(f"{m}p{e}")
            vals += [v, -v]
    x = np.array(vals, np.float64)
    y = x[::-1].copy()
    qs = [3.0, float.fromhex("0x1.5555555555555p-2"), float.fromhex("0x1.fffffffffffffp+0"),
          float.fromhex("0x1.0000000000001p+0"), 0.5, 2.0 ** -52, 2.0 ** 52, 2.0 ** -1022 * 3,
          float.fromhex("0x1.8p-1023")]
    for q in qs:
        for op in ("scale", "triad"):
            want = oracle.apply(op, x, y, q)
            for mm in (1, 2):
                got = _run_op(target, dict(variant=sx.SX_VARIANT_VECTOR, threads=128, vec_bytes=16,
                                           unroll=1, fp64_mul=mm), op, x, y, q, np.float64)
                ok = ~np.isnan(want)
                assert_bitwise(got[ok], want[ok], f"{op} q={q!r} mm={mm}")


@pytest.mark.parametrize("mm", [0, 1, 2])
def test_fused_product_units(target, mm):
    e = sx.sx_executor_create(target, sx.SX_PAR, dict(variant=sx.SX_VARIANT_VECTOR, fp64_mul=mm))
    n = 40001
    a, b, c = si.stream_arrays(n, np.float64, base_seed=8)
    ga, gb, gc = _stream_device(target, e, a, b, c, 3.0, 7, fused=True)
    oracle.stream(a, b, c, 3.0, 7)
    assert_bitwise(ga, a)
    assert_bitwise(gb, b)
    assert_bitwise(gc, c)
    sx.sx_executor_destroy(e)


@pytest.mark.parametrize("n", [1, 63, 1000, 18944, 18945, 40001, 151552, 151553])
def test_fused_launch_shapes_by_size(target, executor, n):
    """The fused kernel's launch shape and default product unit change with the elements per SM
    (one element per thread and the FP64 pipe up to 128 per SM, the integer units up to 1024 per
    SM, vectors beyond); every shape gives the oracle's bits, around each boundary (148 SMs)."""
    a, b, c = si.stream_arrays(n, np.float64, base_seed=9)
    ga, gb, gc = _stream_device(target, executor, a, b, c, 3.0, 9, fused=True)
    oracle.stream(a, b, c, 3.0, 9)
    for g, w, name in ((ga, a, "a"), (gb, b, "b"), (gc, c, "c")):
        assert_bitwise(g, w, f"{name}, n={n}")


def test_device_failure_path_selftest():
    """A kernel's bounded wait that runs out reports SX_ERR_DEVICE at the next synchronisation
    and leaves the context usable (no trap, no hang: the wait is limited to 2 ms)."""
    t = sx.sx_target_create(0)
    e = sx.sx_executor_create(t, sx.SX_PAR)
    try:
        sx.sx_target_selftest(t, 2000)
        with pytest.raises(sx.SxError) as ei:
            sx.sx_target_synchronize(t)
        assert ei.value.status == sx.SX_ERR_DEVICE
        sx.sx_target_synchronize(t)  # the word was cleared
        x, y = _inputs(1000, np.float64, 9)
        dx, dy, do = to_device(t, x), to_device(t, y), empty(t, np.float64, 1000)
        sx.sx_transform_triad(e, dx, dy, do, 3.0)
        assert_bitwise(to_host(do), oracle.triad(x, y, 3.0))
        for a in (dx, dy, do):
            sx.sx_free(a)
        with pytest.raises(sx.SxError):
            sx.sx_target_selftest(t, 0)
    finally:
        sx.sx_executor_destroy(e)
        sx.sx_target_destroy(t)


def test_stream_host_pipelined_chunks(target, executor):
    """End to end over several 32 MiB chunks on the pipeline streams, ragged last chunk, with the
    target's own stream busy before and used after."""
    for dt in (np.float64, np.float32):
        n = (9 << 20) + 12345
        a, b, c = si.stream_arrays(n, dt, base_seed=23)
        ha, hb, hc = a.copy(), b.copy(), c.copy()
        da, db, dc = (empty(target, dt, n) for _ in range(3))
        sx.sx_bulk_construct(da, 7.0)  # queued on the target's stream before the pipeline
        sx.sx_stream_host(executor, ha.ctypes.data, hb.ctypes.data, hc.ctypes.data, da, db, dc, 3.0, 2)
        oracle.stream(a, b, c, 3.0, 2)
        assert_bitwise(ha, a, "a")
        assert_bitwise(hb, b, "b")
        assert_bitwise(hc, c, "c")
        assert_bitwise(to_host(da), a, "device a")
        for h in (da, db, dc):
            sx.sx_free(h)


def test_passes_on_several_targets_at_once():
    """Asynchronous execution on several targets (one stream each): independent STREAM sets
    enqueued pass by pass with PAR_TASK executors, futures on each target, then waited for; every
    set equals its own serial oracle run, and a set borrowed by another target's executor gives
    the same bits."""
    sets, n, passes = 3, 100003, 4
    tgts = [sx.sx_target_create(0) for _ in range(sets)]
    execs = [sx.sx_executor_create(t, sx.SX_PAR_TASK) for t in tgts]
    host = [si.stream_arrays(n, np.float64, base_seed=40 + k) for k in range(sets)]
    dev = [[to_device(tgts[k], h) for h in host[k]] for k in range(sets)]
    for _ in range(passes):
        for k in range(sets):
            sx.sx_stream_iter(execs[k], *dev[k], 3.0, 1)
    futs = [sx.sx_execute_async(execs[k], sx.SX_OP_COPY, dev[k][0], None, dev[k][2], 0.0) for k in range(sets)]
    for f in futs:
        sx.sx_future_wait(f, 10000)
        sx.sx_future_destroy(f)
    for k in range(sets):
        a, b, c = (h.copy() for h in host[k])
        oracle.stream(a, b, c, 3.0, passes)
        c = a.copy()
        for got, want in zip(dev[k], (a, b, c)):
            assert_bitwise(to_host(got), want, f"set {k}")
    # the same memory through another target's executor
    ptrs = [sx.sx_array_data(x)[0] for x in dev[1]]
    borrowed = [sx.sx_array_wrap(tgts[0], sx.SX_F64, p, n) for p in ptrs]
    a, b, c = (to_host(x) for x in dev[1])
    sx.sx_stream_iter(execs[0], *borrowed, 3.0, 2)
    sx.sx_executor_wait(execs[0])
    oracle.stream(a, b, c, 3.0, 2)
    for got, want in zip(dev[1], (a, b, c)):
        assert_bitwise(to_host(got), want, "borrowed")
    for x in borrowed + [x for d in dev for x in d]:
        sx.sx_free(x)
    for e in execs:
        sx.sx_executor_destroy(e)
    for t in tgts:
        sx.sx_target_destroy(t)


def test_tuner_lookup_takes_the_nearest_bucket(tmp_path):
    """A table with triad FP64 entries at log2 buckets 20 and 24 only: sizes in between take the
    nearer entry (the larger on a tie), sizes outside take the closest end, other ops none; an
    AUTO executor launches with the looked-up shape and stays exact."""
    import json
    t = sx.sx_target_create(0)
    name = sx.sx_target_info_get(t)["name"]

    def entry(bucket, threads):
        return {"device": name, "op": sx.SX_OP_TRIAD, "dtype": sx.SX_F64, "bucket": bucket, "variant": 1,
                "threads": threads, "blocks_per_sm": 0, "vec_bytes": 16, "unroll": 1, "cache_hint": 0,
                "tile_bytes": 0, "stages": 0, "fp64_mul": 2}
    path = tmp_path / "table.json"
    path.write_text(json.dumps({"ops": [entry(20, 128), entry(24, 512)], "batch": []}))
    sx.sx_tune_clear()
    try:
        sx.sx_tune_load(str(path))
        for n, threads in ((1 << 10, 128), (1 << 20, 128), (1 << 21, 128), (1 << 22, 512), (1 << 23, 512),
                           (1 << 30, 512)):
            assert sx.sx_tune_lookup(t, sx.SX_OP_TRIAD, sx.SX_F64, n)["threads"] == threads, n
        assert sx.sx_tune_lookup(t, sx.SX_OP_ADD, sx.SX_F64, 1 << 20) is None
        assert sx.sx_tune_lookup(t, sx.SX_OP_TRIAD, sx.SX_F32, 1 << 20) is None
        e = sx.sx_executor_create(t, sx.SX_PAR)
        assert sx.sx_executor_resolve(e, sx.SX_OP_TRIAD, sx.SX_F64, 3 << 20)["threads"] == 128  # bucket 21
        assert sx.sx_executor_resolve(e, sx.SX_OP_TRIAD, sx.SX_F64, 3 << 21)["threads"] == 512  # 22: a tie
        x, y = _inputs(3 << 21, np.float64, 13)
        dx, dy, do = to_device(t, x), to_device(t, y), empty(t, np.float64, x.size)
        sx.sx_execute(e, sx.SX_OP_TRIAD, dx, dy, do, 3.0)
        assert_bitwise(to_host(do), oracle.triad(x, y, 3.0), "auto from the table")
        for h in (dx, dy, do):
            sx.sx_free(h)
        sx.sx_executor_destroy(e)
    finally:
        sx.sx_tune_clear()
        sx.load_shipped_tune_table()
        sx.sx_target_destroy(t)


def test_c_client_closed_form(tmp_path):
    """A plain C11 program (tests/c_abi_program.c) runs STREAM's closed form through the C ABI."""
    import subprocess
    from test_abi import build_c_client
    r = subprocess.run([build_c_client(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "closed form ok" in r.stdout, (r.returncode, r.stdout, r.stderr)


def test_target_on_torchs_default_stream_is_ordered_with_torch():
    """torch names its default (legacy) stream 0; the target borrows it as cudaStreamLegacy, so
    a library call enqueued after an asynchronous torch copy reads the copied data, and torch
    reads the library's result after it."""
    import torch
    import paper_2206_06302_b300 as pkg
    assert torch.cuda.current_stream().cuda_stream == 0
    t = pkg.target_on_torch_stream(0)
    assert sx.sx_target_stream(t) == pkg.CUDA_STREAM_LEGACY
    e = sx.sx_executor_create(t, sx.SX_PAR_TASK)
    n = 1 << 26
    hx = torch.from_numpy(si.uniform(77, n, np.float64)).pin_memory()
    hy = torch.from_numpy(si.uniform(78, n, np.float64)).pin_memory()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    o = torch.zeros_like(x)
    torch.cuda.synchronize()
    x.copy_(hx, non_blocking=True)  # ~10 ms of copies still in flight when the triad is enqueued
    y.copy_(hy, non_blocking=True)
    wx, wy, wo = (pkg.wrap_tensor(t, v) for v in (x, y, o))
    sx.sx_execute_async(e, sx.SX_OP_TRIAD, wx, wy, wo, 3.0, future=False)
    got = o.cpu().numpy()  # torch's stream: after the triad
    assert_bitwise(got, oracle.triad(hx.numpy(), hy.numpy(), 3.0), "ordered with torch")
    for w in (wx, wy, wo):
        sx.sx_free(w)
    sx.sx_executor_destroy(e)
    sx.sx_target_destroy(t)


def test_programmatic_launches_keep_order_with_torch_kernels():
    """Each VECTOR kernel is launched as a programmatic dependent of the kernel before it on the
    stream.  A chain on one non-default stream that alternates library kernels (scale, triad,
    copy, add) with torch kernels, every step reading what the step before wrote, gives the
    serial result bit for bit, for one-block, multi-block and multi-wave arrays."""
    import torch
    import paper_2206_06302_b300 as pkg
    s = torch.cuda.Stream()
    t = pkg.target_on_torch_stream(0, s)
    e = sx.sx_executor_create(t, sx.SX_PAR_TASK)
    for n in (1000, 65537, (1 << 22) + 3):
        hx = si.uniform(si.array_seed(4242, 0, n), n, np.float64)
        with torch.cuda.stream(s):
            x = torch.from_numpy(hx).to("cuda", non_blocking=False)
            y, z = torch.empty_like(x), torch.empty_like(x)
            wx, wy, wz = (pkg.wrap_tensor(t, v) for v in (x, y, z))
            rx = hx.copy()
            for _ in range(12):
                sx.sx_execute_async(e, sx.SX_OP_SCALE, wx, None, wy, 3.0, future=False)  # y = 3x
                torch.sub(y, 1.0, out=x)                                                # x = y - 1
                sx.sx_execute_async(e, sx.SX_OP_TRIAD, wx, wy, wz, 3.0, future=False)  # z = x + 3y
                torch.mul(z, 0.25, out=x)                                               # x = z / 4
                sx.sx_execute_async(e, sx.SX_OP_COPY, wx, None, wy, 0.0, future=False)  # y = x
                sx.sx_execute_async(e, sx.SX_OP_ADD, wx, wy, wz, 0.0, future=False)     # z = x + y
                torch.sub(z, y, out=x)                                                  # x = z - y
                ry = oracle.scale(rx, 3.0)
                rx = ry - 1.0
                rz = oracle.triad(rx, ry, 3.0)
                rx = rz * 0.25
                ry = oracle.copy(rx)
                rz = oracle.add(rx, ry)
                rx = rz - ry
            got = [v.cpu().numpy() for v in (x, y, z)]
        for g, w, name in zip(got, (rx, ry, rz), "xyz"):
            assert_bitwise(g, w, f"{name}, n={n}")
        for w in (wx, wy, wz):
            sx.sx_free(w)
    sx.sx_executor_destroy(e)
    sx.sx_target_destroy(t)


UPPER_SRC = """
__device__ sx_t sx_fn(sx_t c) {
    return (c >= 'a' && c <= 'z') ? (sx_t)(c - ('a' - 'A')) : c;
}
"""


def test_transform_with_a_callable_given_as_source(target, executor):
    """Any device callable (Section 4.2), compiled at run time: Listing 3's to_upper given as
    source equals the oracle's; binary64 and binary32 expressions round each operation once
    (no contraction), in place as well; the compiled callable is reused; a callable that does not
    compile is refused with the compiler's message."""
    text = np.frombuffer(b"hello, world " + bytes(range(256)) * 13 + b"tail", np.uint8).copy()
    ds, do = to_device(target, text), empty(target, np.uint8, text.size)
    for _ in range(2):  # the second call takes the compiled callable from the cache
        sx.sx_transform_src(executor, UPPER_SRC, ds, do)
        assert_bitwise(to_host(do), oracle.to_upper(text), "to_upper from source")
    for h in (ds, do):
        sx.sx_free(h)
    n = 100003
    x64 = _inputs(n, np.float64, 21)[0]
    dx = to_device(target, x64)
    do = empty(target, np.float64, n)
    sx.sx_transform_src(executor, "__device__ sx_t sx_fn(sx_t x) { return x * 2.5 + 1.0; }", dx, do)
    assert_bitwise(to_host(do), np.add(np.multiply(x64, 2.5), 1.0), "binary64 x*2.5+1")
    sx.sx_transform_src(executor, "__device__ sx_t sx_fn(sx_t x) { return x * x; }", dx, dx)  # in place
    assert_bitwise(to_host(dx), np.multiply(x64, x64), "binary64 x*x in place")
    for h in (dx, do):
        sx.sx_free(h)
    x32 = _inputs(n, np.float32, 22)[0]
    dx, do = to_device(target, x32), empty(target, np.float32, n)
    sx.sx_transform_src(executor, "__device__ sx_t sx_fn(sx_t x) { return x * x - 0.5f; }", dx, do)
    want = np.subtract(np.multiply(x32, x32, dtype=np.float32), np.float32(0.5), dtype=np.float32)
    assert_bitwise(to_host(do), want, "binary32 x*x-0.5")
    with pytest.raises(sx.SxError) as ei:
        sx.sx_transform_src(executor, "__device__ sx_t sx_fn(sx_t x) { return undefined_name; }", dx, do)
    assert ei.value.status == sx.SX_ERR_INVALID and "undefined_name" in str(ei.value)
    for h in (dx, do):
        sx.sx_free(h)


def test_cpp_layer_closed_form(tmp_path):
    """The header-only C++ layer (include/sx.hpp): STREAM as algorithm calls under par.on(exec)
    on allocator-placed vectors, then the library's pass loop, reaches the closed form exactly."""
    import subprocess
    from test_abi import build_cpp_client
    r = subprocess.run([build_cpp_client(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "closed form ok" in r.stdout, (r.returncode, r.stdout, r.stderr)


@pytest.mark.parametrize("n", [1 << 16, 1 << 20])
def test_pass_tuner(n):
    """sx_tune_pass times the four kernels together in a STREAM pass: each shape it returns is the
    kernel's starting shape (the shipped table's entry) with at most the cache hint changed, it is
    stored under (device, op, type, log2 n) and found again by sx_tune_lookup, an AUTO executor's
    passes (sx_stream_iter) launch with it, and three passes from seeded inputs with a ragged
    tail equal the oracle's bit for bit."""
    t = sx.sx_target_create(0)
    try:
        for dt, code in ((np.float64, sx.SX_F64), (np.float32, sx.SX_F32)):
            e = sx.sx_executor_create(t, sx.SX_PAR)
            start = [sx.sx_executor_resolve(e, op, code, n) for op in OPS.values()]
            best, gbs = sx.sx_tune_pass(t, code, n)
            assert gbs > 0
            for k, op in enumerate(OPS.values()):
                assert best[k]["cache_hint"] in (0, 1)
                if start[k]["variant"] != sx.SX_VARIANT_VECTOR:
                    assert best[k] == start[k]
                assert {f: v for f, v in best[k].items() if f != "cache_hint"} == \
                    {f: v for f, v in start[k].items() if f != "cache_hint"}
                assert sx.sx_tune_lookup(t, op, code, n) == best[k]
                assert sx.sx_executor_resolve(e, op, code, n + 37) == best[k]
            a, b, c = si.stream_arrays(n + 37, dt, base_seed=31)
            da, db, dc = to_device(t, a), to_device(t, b), to_device(t, c)
            sx.sx_stream_iter(e, da, db, dc, 3.0, 3)
            oracle.stream(a, b, c, 3.0, 3)
            for got, want, nm in zip((da, db, dc), (a, b, c), "abc"):
                assert_bitwise(to_host(got), want, f"pass-tuned {nm} {dt.__name__} n={n}")
            for h in (da, db, dc):
                sx.sx_free(h)
            sx.sx_executor_destroy(e)
    finally:
        sx.sx_tune_clear()
        sx.load_shipped_tune_table()
        sx.sx_target_destroy(t)


def test_pass_tuner_keeps_bulk_copy_shapes(tmp_path):
    """A kernel whose table entry is of a bulk-copy family (no cache hint) keeps its shape through
    sx_tune_pass, and the pass under the result still equals the oracle's bit for bit."""
    import json
    n = 1 << 16
    t = sx.sx_target_create(0)
    try:
        path = str(tmp_path / "table.json")
        sx.sx_tune_save(path)
        table = json.load(open(path))
        bulk = dict(variant=sx.SX_VARIANT_BULK, threads=256, blocks_per_sm=1, vec_bytes=0, unroll=0,
                    cache_hint=0, tile_bytes=16384, stages=3, fp64_mul=2, reserved=0)
        for e in table["ops"]:
            if e["op"] == sx.SX_OP_SCALE and e["dtype"] == sx.SX_F64 and e["bucket"] == 16:
                e.update({k: v for k, v in bulk.items() if k != "reserved"})
        json.dump(table, open(path, "w"))
        sx.sx_tune_load(path)
        assert sx.sx_tune_lookup(t, sx.SX_OP_SCALE, sx.SX_F64, n) == bulk
        best, _ = sx.sx_tune_pass(t, sx.SX_F64, n)
        assert best[1] == bulk and sx.sx_tune_lookup(t, sx.SX_OP_SCALE, sx.SX_F64, n) == bulk
        e = sx.sx_executor_create(t, sx.SX_PAR)
        a, b, c = si.stream_arrays(n + 5, np.float64, base_seed=32)
        da, db, dc = to_device(t, a), to_device(t, b), to_device(t, c)
        sx.sx_stream_iter(e, da, db, dc, 3.0, 2)
        oracle.stream(a, b, c, 3.0, 2)
        for got, want, nm in zip((da, db, dc), (a, b, c), "abc"):
            assert_bitwise(to_host(got), want, f"pass with a BULK scale: {nm}")
        for h in (da, db, dc):
            sx.sx_free(h)
        sx.sx_executor_destroy(e)
    finally:
        sx.sx_tune_clear()
        sx.load_shipped_tune_table()
        sx.sx_target_destroy(t)


@pytest.mark.parametrize("n", [1 << 16, 1 << 20])
def test_per_op_autotuner_search(tmp_path, n):
    """sx_tune searches the launch shapes of the three families for each of the four kernels and
    both types: the shape it returns is valid (an executor fixed to it resolves to it unchanged),
    it is stored under (device, op, type, log2 n) and found again by sx_tune_lookup, an AUTO
    executor launches with it, the results under it equal the oracle's bit for bit (with a
    ragged tail: n + 37 is in the same log2 bucket), and the table round-trips through
    sx_tune_save / sx_tune_load."""
    t = sx.sx_target_create(0)
    sx.sx_tune_clear()
    found = {}
    try:
        for dt, code in ((np.float64, sx.SX_F64), (np.float32, sx.SX_F32)):
            for name, op in OPS.items():
                best, gbs = sx.sx_tune(t, op, code, n)
                assert gbs > 0 and best["variant"] in (sx.SX_VARIANT_VECTOR, sx.SX_VARIANT_BULK,
                                                       sx.SX_VARIANT_TMA), best
                fixed = sx.sx_executor_create(t, sx.SX_PAR, best)  # refused if the shape were invalid
                assert sx.sx_executor_resolve(fixed, op, code, n) == best
                sx.sx_executor_destroy(fixed)
                assert sx.sx_tune_lookup(t, op, code, n) == best
                assert sx.sx_tune_lookup(t, op, code, n + 37) == best
                e = sx.sx_executor_create(t, sx.SX_PAR)
                try:
                    assert sx.sx_executor_resolve(e, op, code, n + 37) == best
                    x, y = _inputs(n + 37, dt, 29)
                    dx, dy, do = to_device(t, x), to_device(t, y), empty(t, dt, x.size)
                    sx.sx_execute(e, op, dx, dy, do, 3.0)
                    assert_bitwise(to_host(do), oracle.apply(name, x, y, 3.0), f"tuned {name} {dt.__name__} n={n}")
                    assert sx.sx_array_guard_ok(do)
                    for h in (dx, dy, do):
                        sx.sx_free(h)
                finally:
                    sx.sx_executor_destroy(e)
                found[(op, code)] = best
        path = str(tmp_path / "tuned.json")
        sx.sx_tune_save(path)
        sx.sx_tune_clear()
        assert sx.sx_tune_lookup(t, sx.SX_OP_TRIAD, sx.SX_F64, n) is None
        sx.sx_tune_load(path)
        for (op, code), best in found.items():
            assert sx.sx_tune_lookup(t, op, code, n) == best
    finally:
        sx.sx_tune_clear()
        sx.load_shipped_tune_table()
        sx.sx_target_destroy(t)
