"""Host-side logic of the multi-GPU (weak scaling) bench path, with two gloo ranks on CPU: the
job's time is the slowest rank's, the throughput sums the ranks' work, every rank draws its own
arrays, and the reference arm prints only on rank 0."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

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
