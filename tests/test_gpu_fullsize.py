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
