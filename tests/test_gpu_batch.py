"""GPU parity of the persistent batched launcher (bulk_execute over many instances) and of its
one-launch-per-instance baseline: every instance's output must equal the oracle's bit for bit,
whatever the tile size, block shape or vector width, with ragged and misaligned instances."""
import numpy as np
import pytest

import oracle
import paper_2206_06302_b300 as sx
import stream_inputs as si
from gpu_util import assert_bitwise

pytestmark = pytest.mark.gpu

OPN = {sx.SX_OP_COPY: "copy", sx.SX_OP_SCALE: "scale", sx.SX_OP_ADD: "add", sx.SX_OP_TRIAD: "triad"}


class Workload:
    """`count` instances carved from one device buffer; some start off the vector alignment."""

    def __init__(self, count, seed, lo_exp=0, hi_exp=16, with_seed_items=True):
        import torch
        ops = [sx.SX_OP_COPY, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_TRIAD]
        if with_seed_items:
            ops.append(sx.SX_OP_SEED)
        lens = si.log_uniform_lengths(si.word_scalar(seed, 1), count, lo_exp, hi_exp)
        opi = si.words(si.word_scalar(seed, 2), count) % np.uint64(len(ops))
        dti = si.words(si.word_scalar(seed, 3), count) % np.uint64(2)
        offs = si.words(si.word_scalar(seed, 4), count) % np.uint64(4)
        self.specs = []
        total = 0
        for k in range(count):
            op = ops[int(opi[k])]
            dt = np.float64 if dti[k] else np.float32
            es = np.dtype(dt).itemsize
            n = int(lens[k])
            off = int(offs[k]) * es if k % 3 == 0 else 0  # every third instance misaligned
            mixed = k % 5 == 1  # and every fifth has arrays misaligned differently
            regions = []
            for j in range(3):
                total = (total + 255) // 256 * 256 + (j * es if mixed else off)
                regions.append(total)
                total += n * es
            self.specs.append(dict(op=op, dt=dt, n=n, regions=regions, q=[3.0, -0.7, 1.5][k % 3],
                                   seed=int(si.word_scalar(seed, 1000 + k)), base=k * 17))
        self.buf = torch.zeros(total + 256, dtype=torch.uint8, device="cuda")
        self.base = self.buf.data_ptr()
        self.host_in = []
        import torch as _t
        for k, s in enumerate(self.specs):
            x = si.uniform(si.array_seed(seed, 0, k), s["n"], s["dt"])
            y = si.uniform(si.array_seed(seed, 1, k), s["n"], s["dt"])
            self.host_in.append((x, y))
            for arr, r in ((x, s["regions"][0]), (y, s["regions"][1])):
                nb = arr.nbytes
                self.buf[r:r + nb] = _t.from_numpy(arr.view(np.uint8)).cuda()
        _t.cuda.synchronize()

    def items(self):
        out = []
        for s in self.specs:
            r = s["regions"]
            out.append(sx.sx_batch_item(
                op=s["op"], dtype=sx.SX_F64 if s["dt"] == np.float64 else sx.SX_F32, n=s["n"],
                x=self.base + r[0], y=self.base + r[1], out=self.base + r[2],
                q=s["q"] if s["op"] != sx.SX_OP_SEED else -1.0, q2=1.0 if s["op"] == sx.SX_OP_SEED else 0.0,
                seed=s["seed"], index_base=s["base"]))
        return out

    def clear_outputs(self):
        for s in self.specs:
            r = s["regions"][2]
            self.buf[r:r + s["n"] * np.dtype(s["dt"]).itemsize] = 0xEE

    def check(self, what):
        import torch
        torch.cuda.synchronize()
        h = self.buf.cpu().numpy()
        for k, s in enumerate(self.specs):
            dt, n = s["dt"], s["n"]
            r = s["regions"][2]
            got = h[r:r + n * np.dtype(dt).itemsize].view(dt)
            x, y = self.host_in[k][0][:n], self.host_in[k][1][:n]
            if s["op"] == sx.SX_OP_SEED:
                want = si.uniform(s["seed"], n, dt, -1.0, 1.0, start=s["base"])
            else:
                want = oracle.apply(OPN[s["op"]], x, y, s["q"])
            assert_bitwise(got, want, f"{what}: instance {k} ({s['op']}, {dt.__name__}, n={n})")


CFGS = [None,
        dict(chunk_bytes=16384, threads=128, blocks_per_sm=1, vec_bytes=16),
        dict(chunk_bytes=65536, threads=256, blocks_per_sm=8, vec_bytes=32),
        dict(chunk_bytes=1 << 20, threads=1024, blocks_per_sm=2, vec_bytes=32)]


@pytest.mark.parametrize("cfg", range(len(CFGS)))
def test_batch_matches_oracle(target, cfg):
    w = Workload(300, seed=11)
    b = sx.sx_batch_create(target, w.items(), CFGS[cfg])
    for rep in range(2):  # the captured graph replays
        w.clear_outputs()
        sx.sx_batch_launch(b)
        sx.sx_target_synchronize(target)
        w.check(f"graph launch {rep}")
    sx.sx_batch_destroy(b)


def test_percall_baseline_matches_oracle(target):
    w = Workload(120, seed=12)
    b = sx.sx_batch_create(target, w.items())
    w.clear_outputs()
    sx.sx_batch_launch_percall(b)
    sx.sx_target_synchronize(target)
    w.check("per-call")
    sx.sx_batch_destroy(b)


def test_completion_recording(target):
    w = Workload(64, seed=13, lo_exp=10, hi_exp=20)
    b = sx.sx_batch_create(target, w.items())
    sx.sx_batch_set_record(b, True)
    for launch in (sx.sx_batch_launch, sx.sx_batch_launch_percall):
        w.clear_outputs()
        launch(b)
        t = sx.sx_batch_completion_ns(b, 64)
        w.check(launch.__name__)
        assert all(v > 0 for v in t) and max(t) < 5e9
    sx.sx_batch_destroy(b)


def test_items_run_shortest_first(target):
    """Both launch kinds run the items in increasing STREAM bytes (equal sizes in the caller's
    order).  Per call: completion times, taken in stream order, rise along that order.  One launch,
    a grid of one block per SM walking small tiles: the smallest half of the items is done before
    any of the ten largest (their tiles are listed ~100 grid rounds apart)."""
    w = Workload(200, seed=14, lo_exp=8, hi_exp=20)
    items = w.items()
    arrays = {sx.SX_OP_COPY: 2, sx.SX_OP_SCALE: 2, sx.SX_OP_ADD: 3, sx.SX_OP_TRIAD: 3, sx.SX_OP_SEED: 1}
    nbytes = [arrays[s["op"]] * s["n"] * np.dtype(s["dt"]).itemsize for s in w.specs]
    order = sorted(range(len(items)), key=lambda k: nbytes[k])  # stable: ties keep the caller's order
    b = sx.sx_batch_create(target, items, dict(chunk_bytes=16384, threads=128, blocks_per_sm=1, vec_bytes=16))
    sx.sx_batch_set_record(b, True)
    w.clear_outputs()
    sx.sx_batch_launch_percall(b)
    t = np.asarray(sx.sx_batch_completion_ns(b, len(items)), dtype=np.float64)
    w.check("per-call, shortest first")
    assert np.all(np.diff(t[order]) >= 0), "per-call items did not complete in the shortest-first order"
    w.clear_outputs()
    sx.sx_batch_launch(b)
    t = np.asarray(sx.sx_batch_completion_ns(b, len(items)), dtype=np.float64)
    w.check("graph, shortest first")
    assert t[order[:100]].max() < t[order[-10:]].min()
    sx.sx_batch_destroy(b)


def test_first_round_runs_first_whatever_blocks_per_sm_asks(target):
    """The persistent grid is capped at the blocks the SMs hold at once: with 2500 one-tile items
    ahead of four large ones and a shape asking for more blocks than fit (128 threads x 16 per SM),
    every small item is done within the first rounds, early in the launch.  (A block left waiting
    for a free SM starts only when a resident block has finished all of its tiles, so the small
    items it owns would be done about halfway through.)  The results equal the oracle's."""
    import torch
    rng = np.random.default_rng(15)
    small = [256] * 2500
    large = [1 << 22] * 4
    lens = small + large
    offs, total = [], 0
    for n in lens:
        r = []
        for _ in range(3):
            total = (total + 255) // 256 * 256
            r.append(total)
            total += n * 8
        offs.append(r)
    buf = torch.zeros(total, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    host = []
    for n, o in zip(lens, offs):
        x, y = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
        host.append((x, y))
        buf[o[0]:o[0] + 8 * n] = torch.from_numpy(x.view(np.uint8)).cuda()
        buf[o[1]:o[1] + 8 * n] = torch.from_numpy(y.view(np.uint8)).cuda()
    items = [sx.sx_batch_item(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=n, x=base + o[0], y=base + o[1],
                              out=base + o[2], q=3.0) for n, o in zip(lens, offs)]
    b = sx.sx_batch_create(target, items, dict(chunk_bytes=16384, threads=128, blocks_per_sm=16, vec_bytes=32))
    cfg, _, _ = sx.sx_batch_info(b)
    assert 1 <= cfg["blocks_per_sm"] < 16 and cfg["threads"] == 128  # as it runs: capped
    sx.sx_batch_set_record(b, True)
    sx.sx_batch_launch(b)
    t = np.asarray(sx.sx_batch_completion_ns(b, len(items)), dtype=np.float64)
    assert t[:2500].max() < 0.25 * t.max(), (t[:2500].max(), t.max())
    h = buf.cpu().numpy()
    for k in list(range(0, 2500, 97)) + [2500, 2503]:
        n, o = lens[k], offs[k]
        got = h[o[2]:o[2] + 8 * n].view(np.float64)
        assert_bitwise(got, oracle.apply("triad", host[k][0], host[k][1], 3.0), f"item {k}")
    sx.sx_batch_destroy(b)


def test_empty_and_zero_length_items(target):
    b = sx.sx_batch_create(target, [])
    sx.sx_batch_launch(b)
    sx.sx_target_synchronize(target)
    sx.sx_batch_destroy(b)
    w = Workload(10, seed=14)
    items = w.items()
    items[3].n = 0
    w.specs[3]["n"] = 0
    b = sx.sx_batch_create(target, items)
    sx.sx_batch_launch(b)
    w.check("with an empty item")
    sx.sx_batch_destroy(b)


def test_batch_autotune_keeps_results(target):
    w = Workload(200, seed=15, lo_exp=8, hi_exp=18, with_seed_items=False)
    b = sx.sx_batch_create(target, w.items())
    best, ms = sx.sx_tune_batch(b)
    assert ms > 0 and best["chunk_bytes"] >= 16384
    w.clear_outputs()
    sx.sx_batch_launch(b)
    w.check("after tuning")
    cfg, tiles, nbytes = sx.sx_batch_info(b)
    assert cfg == best and tiles > 0 and nbytes > 0
    sx.sx_batch_destroy(b)


def test_bad_items_are_rejected(target):
    it = sx.sx_batch_item(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=10, x=None, y=None, out=None)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_batch_create(target, [it])
    assert ei.value.status == sx.SX_ERR_INVALID
    it = sx.sx_batch_item(op=9, dtype=sx.SX_F64, n=10)
    with pytest.raises(sx.SxError):
        sx.sx_batch_create(target, [it])
    with pytest.raises(sx.SxError):
        sx.sx_batch_create(target, [], dict(chunk_bytes=100, threads=256, blocks_per_sm=1, vec_bytes=32))


@pytest.mark.parametrize("vec", [16, 32])
def test_batch_products_on_every_bit_pattern(target, vec):
    """FP64 SCALE and TRIAD items on random bit patterns (zeros, subnormals, values near the
    overflow threshold, infinities, NaNs) with scalars that take each product variant (short and
    long significands, subnormal, zero, infinite): every output equals the oracle wherever the
    oracle's result is not a NaN, and is a NaN exactly where it is (a generated NaN's sign and
    payload are unspecified).  Items start at different offsets of the vector alignment."""
    import torch
    n = 20011
    x = si.words(71, n).view(np.float64).copy()
    y = si.words(72, n).view(np.float64).copy()
    qs = [3.0, -0.1, 1.0, 2.0 ** -1022, 5e-324, 1.7976931348623157e308, 1e300, -7.5, float("inf"), 0.0]
    narr = 2 + 2 * len(qs)
    buf = torch.zeros(narr * (n * 8 + 512), dtype=torch.uint8, device="cuda")  # 512: alignment + offset
    base = buf.data_ptr()
    at = [0]

    def put(arr, off):
        at[0] = (at[0] + 255) // 256 * 256 + 8 * off
        p = at[0]
        buf[p:p + arr.nbytes] = torch.from_numpy(arr.view(np.uint8)).cuda()
        at[0] += arr.nbytes
        return p

    px, py = put(x, 1), put(y, 1)
    items, outs = [], []
    for k, q in enumerate(qs):
        for op in (sx.SX_OP_SCALE, sx.SX_OP_TRIAD):
            po = put(np.zeros(n), 1 if k % 2 else 3)
            items.append(sx.sx_batch_item(op=op, dtype=sx.SX_F64, n=n, x=base + px, y=base + py,
                                          out=base + po, q=q))
            outs.append((po, op, q))
    torch.cuda.synchronize()
    b = sx.sx_batch_create(target, items, dict(chunk_bytes=16384, threads=256, blocks_per_sm=2, vec_bytes=vec))
    sx.sx_batch_launch(b)
    sx.sx_target_synchronize(target)
    sx.sx_batch_destroy(b)
    h = buf.cpu().numpy()
    for po, op, q in outs:
        got = h[po:po + 8 * n].view(np.float64)
        want = oracle.apply(OPN[op], x, y, q)
        ok = ~np.isnan(want)
        assert_bitwise(got[ok], want[ok], f"{OPN[op]} q={q}")
        assert np.array_equal(np.isnan(got), np.isnan(want)), f"{OPN[op]} q={q} NaN positions"


def test_bulk_async_execute_future(target):
    """sx_batch_launch_async (Listing 2's bulk_async_execute): the future completes once every
    item has run, reports the launch's device time, and the outputs equal the oracle's."""
    import torch
    w = Workload(200, seed=14)
    b = sx.sx_batch_create(target, w.items())
    for rep in range(2):
        w.clear_outputs()
        torch.cuda.synchronize()
        f = sx.sx_batch_launch_async(b)
        sx.sx_future_wait(f, 60000)
        assert sx.sx_future_test(f)
        assert 0.0 < sx.sx_future_elapsed_ms(f) < 10000.0
        sx.sx_future_destroy(f)
        w.check(f"async launch {rep}")
    sx.sx_batch_destroy(b)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_batch_launch_async(None)
    assert ei.value.status == sx.SX_ERR_INVALID
