"""GPU parity of the block partition (Section 4.1's block allocator over a vector of targets):
one logical array split into contiguous blocks, each block on a target of its own, constructed
with sx_seed_uniform_at at its offset and run through STREAM passes by that target's executor.

Bar: every block's seeded inputs equal the matching slice of the whole array (and of the host
generator), and the blocks' results put together equal the oracle's passes over the whole
arrays bit for bit (and the one-target run), for part counts that do and do not divide n.  The
blocks run one after another here (one GPU); on several GPUs each would be one rank's."""
import numpy as np
import pytest

import oracle
import paper_2206_06302_b300 as sx
import stream_inputs as si
from gpu_util import assert_bitwise, to_host

pytestmark = pytest.mark.gpu

CODE = {np.float64: sx.SX_F64, np.float32: sx.SX_F32}


def _seeded_block(t, dt, n_block, off, k, base=77):
    a = sx.sx_alloc(t, CODE[dt], n_block)
    sx.sx_seed_uniform_at(a, si.array_seed(base, k, 0), -1.0, 1.0, off)
    return a


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("parts", [2, 3, 5])
def test_blocks_of_one_array_match_the_whole(dt, parts):
    n, passes = (1 << 18) + 37, 3
    whole_in = [si.uniform(si.array_seed(77, k, 0), n, dt) for k in range(3)]
    want = [w.copy() for w in whole_in]
    oracle.stream(*want, 3.0, passes)
    got = [[] for _ in range(3)]
    for part in range(parts):
        off, cnt = sx.sx_block_partition(n, parts, part)
        t = sx.sx_target_create(0)  # the block's own target (a rank's GPU on a multi-GPU node)
        e = sx.sx_executor_create(t, sx.SX_PAR)
        try:
            arrs = [_seeded_block(t, dt, cnt, off, k) for k in range(3)]
            sx.sx_target_synchronize(t)
            for k, a in enumerate(arrs):
                assert_bitwise(to_host(a), whole_in[k][off:off + cnt], f"block {part} input {'abc'[k]}")
            sx.sx_stream_iter(e, *arrs, 3.0, passes)
            for k, a in enumerate(arrs):
                got[k].append(to_host(a))
                assert sx.sx_array_guard_ok(a)
                sx.sx_free(a)
        finally:
            sx.sx_executor_destroy(e)
            sx.sx_target_destroy(t)
    for k in range(3):
        assert_bitwise(np.concatenate(got[k]), want[k], f"{parts} blocks, array {'abc'[k]}")


def test_one_target_run_equals_the_blocks(target, executor):
    """The whole arrays on one target (sx_seed_uniform, index 0) and the same arrays as two
    blocks: identical bits after the passes."""
    n, passes = (1 << 20) + 3, 2
    whole = [sx.sx_alloc(target, sx.SX_F64, n) for _ in range(3)]
    for k, a in enumerate(whole):
        sx.sx_seed_uniform(a, si.array_seed(77, k, 0), -1.0, 1.0)
    sx.sx_stream_iter(executor, *whole, 3.0, passes)
    ref = [to_host(a) for a in whole]
    for a in whole:
        sx.sx_free(a)
    for part in range(2):
        off, cnt = sx.sx_block_partition(n, 2, part)
        arrs = [_seeded_block(target, np.float64, cnt, off, k) for k in range(3)]
        sx.sx_stream_iter(executor, *arrs, 3.0, passes)
        for k, a in enumerate(arrs):
            assert_bitwise(to_host(a), ref[k][off:off + cnt], f"block {part} array {'abc'[k]}")
            sx.sx_free(a)


def test_seed_at_index_overflow_is_refused(target):
    a = sx.sx_alloc(target, sx.SX_F64, 16)
    try:
        with pytest.raises(sx.SxError) as ei:
            sx.sx_seed_uniform_at(a, 1, -1.0, 1.0, (1 << 64) - 8)
        assert ei.value.status == sx.SX_ERR_INVALID
        sx.sx_seed_uniform_at(a, 1, -1.0, 1.0, (1 << 64) - 16)  # the last index is 2^64 - 1: allowed
        sx.sx_target_synchronize(target)
        assert_bitwise(to_host(a), si.uniform(1, 16, np.float64, start=(1 << 64) - 16), "top of the index range")
    finally:
        sx.sx_free(a)
