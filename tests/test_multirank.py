"""Host-side logic of the multi-GPU bench paths, with two gloo ranks on CPU.

Weak scaling (replicas): the job's time is the slowest rank's, the throughput sums the ranks'
work, every rank draws its own arrays, and the reference arm prints only on rank 0.

Block partition (``bench.py --shard``, Section 4.1's block allocator over a vector of targets):
the ranks' blocks tile [0, n) exactly, also when the rank count does not divide n; each rank's
seeded block equals the matching slice of the whole arrays; each block's STREAM passes (the
oracle here, on CPU) equal that slice of the passes over the whole arrays; and the job's time is
the slowest rank's while the throughput counts the whole arrays once."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import stream_inputs as si
    local_ms = [100.0, 250.0][rank]
    gbs, ms = bench.job_throughput(dist, local_ms, 1e9, 10, world, "cpu")
    seeds = [si.array_seed(si.BASE_SEED, k, rank) for k in range(3)]
    out.put((rank, gbs, ms, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gbs, ms, _ in res:
        assert ms == 250.0  # the slowest rank's time, on every rank
        assert gbs == pytest.approx(2 * 1e9 * 10 / 0.25 / 1e9)  # both ranks' bytes
    assert set(res[0][3]).isdisjoint(res[1][3])  # each rank runs its own arrays


def test_single_rank_throughput():
    sys.path.insert(0, ROOT)
    import bench
    gbs, ms = bench.job_throughput(None, 2.0, 4e9, 5, 1, "cpu")
    assert ms == 2.0 and gbs == pytest.approx(4e9 * 5 / 2e-3 / 1e9)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    args = ["--impl", "reference", "--steps", "3", "--warmup", "3", "--ref-n", "4096"]
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main(args) == 0
    assert buf.getvalue() == ""
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main(args) == 0
    line = json.loads(buf.getvalue().strip())
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def _shard_worker(rank, world, port, n, passes, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import paper_2206_06302_b300 as sx
    import stream_inputs as si
    off, cnt = bench.shard_block(sx, n, world, rank)
    # every rank seeds its block by global element index, from the whole arrays' seeds
    arrs = [si.uniform(si.array_seed(si.BASE_SEED, k, 0), cnt, np.float64, start=off) for k in range(3)]
    oracle.stream(*arrs, 3.0, passes)
    local_ms = [100.0, 250.0][rank]
    gbs, ms = bench.job_throughput(dist, local_ms, 10.0 * n * 8, passes, world, "cpu", "strong")
    out.put((rank, off, cnt, [a.copy() for a in arrs], gbs, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_array_into_blocks():
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    import stream_inputs as si
    n, passes = 100003, 3  # odd: the two blocks differ in length
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, n, passes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the blocks tile [0, n) in rank order
    assert res[0][1] == 0 and res[0][2] == (n + 1) // 2
    assert res[1][1] == res[0][2] and res[0][2] + res[1][2] == n
    for rank, off, cnt, arrs, gbs, ms in res:
        assert ms == 250.0  # the slowest rank's time, on every rank
        assert gbs == pytest.approx(10.0 * n * 8 * passes / 0.25 / 1e9)  # the whole arrays, once
    # the blocks' passes, put together, are the passes over the whole arrays, bit for bit
    whole = [si.uniform(si.array_seed(si.BASE_SEED, k, 0), n, np.float64) for k in range(3)]
    oracle.stream(*whole, 3.0, passes)
    for k in range(3):
        got = np.concatenate([res[0][3][k], res[1][3][k]])
        assert np.array_equal(got.view(np.uint64), whole[k].view(np.uint64)), "abc"[k]


def test_block_partition_tiles_every_size():
    """sx_block_partition (host arithmetic): for many n and part counts the blocks are contiguous,
    in order, cover [0, n) exactly, and none is longer than ceil(n / parts)."""
    sys.path.insert(0, ROOT)
    import paper_2206_06302_b300 as sx
    import stream_inputs as si
    for n in (0, 1, 2, 5, 7, 64, 1000, 100003, (1 << 27), (1 << 29) + 7, (1 << 40) + 3):
        for parts in (1, 2, 3, 4, 5, 7, 8, 16):
            at = 0
            for part in range(parts):
                off, cnt = sx.sx_block_partition(n, parts, part)
                assert off == at and cnt <= -(-n // parts)
                at += cnt
            assert at == n
    # seeding by global index: a block drawn at its offset is the slice of the whole array
    for parts in (2, 3, 5):
        n = 4099
        whole = si.uniform(7, n, "float32")
        for part in range(parts):
            off, cnt = sx.sx_block_partition(n, parts, part)
            assert np.array_equal(si.uniform(7, cnt, "float32", start=off), whole[off:off + cnt])
    for bad in ((10, 0, 0), (10, 2, 2), (10, 2, -1), (1 << 63, 2, 0)):
        with pytest.raises(sx.SxError) as ei:
            sx.sx_block_partition(*bad)
        assert ei.value.status == sx.SX_ERR_INVALID
