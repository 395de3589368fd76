"""Parity at the benchmark's full size: STREAM, n = 2^27 per array, seeded uniform [-1, 1) inputs
constructed on the device, q = 3, 100 passes, in binary64 and binary32, with the launch shapes the
benchmark uses.  The oracle recomputes sampled elements one by one (every element's chain of
roundings depends only on its own start values), and the results must agree bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2206_06302_b300 as sx
import stream_inputs as si
from gpu_util import assert_bitwise

pytestmark = pytest.mark.gpu

N = 1 << 27
ITERS = 100


def _sample_indices(n, count, seed):
    rng = np.random.default_rng(seed)
    idx = np.concatenate([np.arange(0, 4096), np.arange(n - 4096, n),
                          rng.integers(0, n, count)])
    return np.unique(idx)


@pytest.mark.parametrize("variant", ["auto", "fused"])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_full_size_stream_sampled(target, dt, variant):
    import torch
    tdt = torch.float64 if dt == np.float64 else torch.float32
    code = sx.SX_F64 if dt == np.float64 else sx.SX_F32
    bufs = [torch.empty(N, dtype=tdt, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    arrs = [sx.sx_array_wrap(target, code, b.data_ptr(), N) for b in bufs]
    seeds = [si.array_seed(si.BASE_SEED, k) for k in range(3)]
    for a, s in zip(arrs, seeds):
        sx.sx_seed_uniform(a, s, -1.0, 1.0)
    e = sx.sx_executor_create(target, sx.SX_PAR_TASK)
    if variant == "fused":
        sx.sx_stream_fused(e, *arrs, 3.0, ITERS)
    else:
        sx.sx_stream_iter(e, *arrs, 3.0, ITERS)
    sx.sx_executor_wait(e)
    idx = _sample_indices(N, 1 << 18, 4)
    tidx = torch.from_numpy(idx.astype(np.int64)).cuda()
    got = [b.index_select(0, tidx).cpu().numpy() for b in bufs]
    a0 = [si.uniform_at(s, idx.astype(np.uint64), dt) for s in seeds]
    oracle.stream(a0[0], a0[1], a0[2], 3.0, ITERS)
    for g, w, name in zip(got, a0, "abc"):
        assert_bitwise(g, w, f"{name} {dt.__name__} {variant}")
    for a in arrs:
        sx.sx_free(a)
    sx.sx_executor_destroy(e)


def _sampled(torch, buf, idx):
    return buf.index_select(0, torch.from_numpy(idx.astype(np.int64)).cuda()).cpu().numpy()


@pytest.mark.parametrize("op", ["copy", "triad"])
def test_beyond_32bit_indices_fp32(target, op):
    """n = 2^32 + 17 binary32 elements per array (17 GB each): indices past 2^32 and a ragged
    tail, sampled against the oracle."""
    import torch
    n = (1 << 32) + 17
    bufs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    x, y, o = (sx.sx_array_wrap(target, sx.SX_F32, b.data_ptr(), n) for b in bufs)
    sx.sx_seed_uniform(x, 31, -1.0, 1.0)
    sx.sx_seed_uniform(y, 32, -1.0, 1.0)
    e = sx.sx_executor_create(target, sx.SX_PAR)
    sx.sx_execute(e, sx.SX_OP_COPY if op == "copy" else sx.SX_OP_TRIAD, x, y, o, 3.0)
    idx = np.unique(np.concatenate([np.arange(0, 64), np.arange(n - 4096, n),
                                    np.arange((1 << 32) - 64, (1 << 32) + 17),
                                    np.random.default_rng(1).integers(0, n, 1 << 16)]))
    xs = si.uniform_at(31, idx.astype(np.uint64), np.float32)
    ys = si.uniform_at(32, idx.astype(np.uint64), np.float32)
    assert_bitwise(_sampled(torch, bufs[0], idx), xs, "seeded x")
    assert_bitwise(_sampled(torch, bufs[2], idx), oracle.apply(op, xs, ys, 3.0), op)
    for a in (x, y, o):
        sx.sx_free(a)
    sx.sx_executor_destroy(e)
    del bufs
    torch.cuda.empty_cache()


FAMILIES = {"auto": None,
            "bulk": dict(variant=sx.SX_VARIANT_BULK, fp64_mul=2),
            "tma": dict(variant=sx.SX_VARIANT_TMA, fp64_mul=2),
            "tma_tensor": dict(variant=sx.SX_VARIANT_TMA_TENSOR, fp64_mul=2)}


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_largest_sweep_size_ragged(target, dt, family):
    """The sweep's largest size plus a ragged tail, every kernel, in the bench's launch shapes
    (auto) and in each bulk-copy family's default shape: persistent blocks walk thousands of
    tiles, and the tensor-map view has 2^21 rows."""
    import torch
    n = (1 << 29) + 7
    tdt = torch.float64 if dt == np.float64 else torch.float32
    code = sx.SX_F64 if dt == np.float64 else sx.SX_F32
    bufs = [torch.empty(n, dtype=tdt, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    x, y, o = (sx.sx_array_wrap(target, code, b.data_ptr(), n) for b in bufs)
    sx.sx_seed_uniform(x, 41, -1.0, 1.0)
    sx.sx_seed_uniform(y, 42, -1.0, 1.0)
    e = sx.sx_executor_create(target, sx.SX_PAR, FAMILIES[family])
    idx = np.unique(np.concatenate([np.arange(0, 64), np.arange(n - 300, n),
                                    np.random.default_rng(2).integers(0, n, 1 << 16)]))
    xs = si.uniform_at(41, idx.astype(np.uint64), dt)
    ys = si.uniform_at(42, idx.astype(np.uint64), dt)
    for name, op in (("copy", 0), ("scale", 1), ("add", 2), ("triad", 3)):
        sx.sx_execute(e, op, x, y, o, 3.0)
        assert_bitwise(_sampled(torch, bufs[2], idx), oracle.apply(name, xs, ys, 3.0), f"{name} {family}")
    for a in (x, y, o):
        sx.sx_free(a)
    sx.sx_executor_destroy(e)
    del bufs
    torch.cuda.empty_cache()


def test_batched_workload_full_size(target):
    """The 4096-instance batched workload (FP64 triad/add, n log-uniform in [2^10, 2^22], ~51 GB)
    in one graph launch with its default shape: every 64th instance compared whole, and sampled
    elements of every instance."""
    inst = si.batched_instances(si.BASE_SEED, 4096)
    offs, total = [], 0
    for _, n in inst:
        r = []
        for _ in range(3):
            total = (total + 255) // 256 * 256
            r.append(total)
            total += n * 8
        offs.append(r)
    buf = sx.sx_alloc(target, sx.SX_U8, total)
    base = sx.sx_array_data(buf)[0]
    seeds = []
    for k, (_, n) in enumerate(inst):
        for j in (0, 1):
            seeds.append(sx.sx_batch_item(op=sx.SX_OP_SEED, dtype=sx.SX_F64, n=n, out=base + offs[k][j],
                                          q=-1.0, q2=1.0, seed=si.array_seed(si.BASE_SEED, j, k)))
    sb = sx.sx_batch_create(target, seeds)
    sx.sx_batch_launch(sb)
    sx.sx_target_synchronize(target)
    sx.sx_batch_destroy(sb)
    code = {"add": sx.SX_OP_ADD, "triad": sx.SX_OP_TRIAD}
    items = [sx.sx_batch_item(op=code[op], dtype=sx.SX_F64, n=n, x=base + o[0], y=base + o[1],
                              out=base + o[2], q=3.0) for (op, n), o in zip(inst, offs)]
    b = sx.sx_batch_create(target, items)
    sx.sx_batch_launch(b)
    sx.sx_target_synchronize(target)
    rng = np.random.default_rng(3)
    for k, (op, n) in enumerate(inst):
        whole = k % 64 == 0
        if whole:
            idx = np.arange(n)
        else:
            idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 8)]))
        got = np.empty(idx.size, np.float64)
        # element reads through borrowed single-element or whole views
        if whole:
            w = sx.sx_array_wrap(target, sx.SX_F64, base + offs[k][2], n)
            sx.sx_copy_d2h(got.ctypes.data, w, n)
            sx.sx_free(w)
        else:
            for m, i in enumerate(idx):
                w = sx.sx_array_wrap(target, sx.SX_F64, base + offs[k][2] + 8 * int(i), 1)
                sx.sx_copy_d2h(got[m:m + 1].ctypes.data, w, 1)
                sx.sx_free(w)
        xs = si.uniform_at(si.array_seed(si.BASE_SEED, 0, k), idx.astype(np.uint64), np.float64)
        ys = si.uniform_at(si.array_seed(si.BASE_SEED, 1, k), idx.astype(np.uint64), np.float64)
        assert_bitwise(got, oracle.apply(op, xs, ys, 3.0), f"instance {k} ({op}, n={n})")
    sx.sx_batch_destroy(b)
    sx.sx_free(buf)
