"""GPU tests of the serving loop: every request's inputs and result are bit-identical to the
request run alone and to the oracle, in continuous-batching and per-call FIFO modes, under
admission pressure; requests that arrive while others run overlap with them."""
import numpy as np
import pytest

import oracle
import paper_2206_06302_b300 as sx
import stream_inputs as si

pytestmark = pytest.mark.gpu

OPN = {sx.SX_OP_COPY: "copy", sx.SX_OP_SCALE: "scale", sx.SX_OP_ADD: "add", sx.SX_OP_TRIAD: "triad"}
NP = {sx.SX_F32: np.float32, sx.SX_F64: np.float64}


def _requests(count, seed, lo_exp=4, hi_exp=18):
    ops = [sx.SX_OP_COPY, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_TRIAD]
    lens = si.log_uniform_lengths(si.word_scalar(seed, 1), count, lo_exp, hi_exp)
    out = []
    for k in range(count):
        out.append(dict(op=ops[k % 4], dtype=sx.SX_F64 if (k // 4) % 2 == 0 else sx.SX_F32,
                        n=int(lens[k]), q=[3.0, -0.25, 1.0 / 3.0][k % 3],
                        seed_x=int(si.word_scalar(seed, 100 + 2 * k)),
                        seed_y=int(si.word_scalar(seed, 101 + 2 * k)), lo=-1.0, hi=1.0))
    return out


def _read(s, rid, which, r):
    dt = NP[r["dtype"]]
    h = np.empty(r["n"], dt)
    sx.sx_server_read(s, rid, which, h.ctypes.data, r["n"])
    return h


def _expected(r):
    dt = NP[r["dtype"]]
    x = si.uniform(r["seed_x"], r["n"], dt, r["lo"], r["hi"])
    y = si.uniform(r["seed_y"], r["n"], dt, r["lo"], r["hi"])
    return x, y, oracle.apply(OPN[r["op"]], x, y, r["q"])


def _check_all(s, ids, reqs, what):
    for rid, r in zip(ids, reqs):
        st = sx.sx_server_wait(s, rid, 60000)
        assert st["state"] == sx.SX_REQ_DONE, (what, rid, st)
        x, y, want = _expected(r)
        got = _read(s, rid, 2, r)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (what, rid, r)
        assert np.array_equal(_read(s, rid, 0, r).view(np.uint8), x.view(np.uint8)), (what, rid)
        if r["op"] in (sx.SX_OP_ADD, sx.SX_OP_TRIAD):
            assert np.array_equal(_read(s, rid, 1, r).view(np.uint8), y.view(np.uint8)), (what, rid)
        sx.sx_server_release(s, rid)


@pytest.mark.parametrize("mode", [sx.SX_SERVE_CONTINUOUS, sx.SX_SERVE_FIFO])
def test_each_request_alone(target, mode):
    s = sx.sx_server_create(target, budget_bytes=1 << 30, mode=mode)
    reqs = _requests(8, seed=3, lo_exp=16, hi_exp=17)
    for r in reqs:
        rid = sx.sx_server_submit(s, **r)
        _check_all(s, [rid], [r], "alone")
    sx.sx_server_destroy(s)


@pytest.mark.parametrize("mode,split", [(sx.SX_SERVE_CONTINUOUS, 0), (sx.SX_SERVE_CONTINUOUS, 1),
                                        (sx.SX_SERVE_FIFO, 0)])
def test_mix_equals_alone(target, mode, split):
    """200 requests of mixed op, type and length arrive together; small step budget and tiles
    make long requests span many steps and share them with short ones (as construct-then-operate
    ranges, or with split_phases in two phases)."""
    reqs = _requests(200, seed=4)
    s = sx.sx_server_create(target, budget_bytes=256 << 20, mode=mode, chunk_bytes=1 << 20,
                            tile_bytes=16384, max_active=64, steps_in_flight=2, split_phases=split)
    ids = [sx.sx_server_submit(s, **r) for r in reqs]
    _check_all(s, ids, reqs, "mix")
    st = sx.sx_server_stats_get(s)
    assert st["completed"] == 200 and st["rejected"] == 0
    assert st["arena_peak"] <= 256 << 20
    if mode == sx.SX_SERVE_CONTINUOUS:
        assert st["steps"] > 1
    sx.sx_server_destroy(s)


@pytest.mark.parametrize("split", [0, 1])
def test_short_requests_run_whole_and_report_early(target, split):
    """Requests that a step takes whole run as one construct-then-operate piece and complete from
    that piece's own report, while the long request sharing their steps goes on in ranges (with
    split_phases only requests within a quarter of the step budget run whole; longer ones run in
    two phases).  Every result is the oracle's."""
    s = sx.sx_server_create(target, budget_bytes=8 << 30, chunk_bytes=1 << 30, split_phases=split)
    long_r = dict(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=1 << 27, q=3.0, seed_x=91, seed_y=92,
                  lo=-1.0, hi=1.0)  # 5 GiB of work: several 1 GiB steps of ~0.15 ms
    mid_r = dict(op=sx.SX_OP_ADD, dtype=sx.SX_F32, n=20 << 20, q=1.0, seed_x=93, seed_y=94,
                 lo=-2.0, hi=0.5)  # 400 MiB of work: over a quarter of the budget, two phases
    shorts = [dict(op=[sx.SX_OP_COPY, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_TRIAD][k % 4],
                   dtype=sx.SX_F64 if k % 2 else sx.SX_F32, n=(1 << 14) + 37 * k, q=-0.5,
                   seed_x=200 + k, seed_y=300 + k, lo=-1.0, hi=1.0) for k in range(16)]
    lid = sx.sx_server_submit(s, **long_r)
    mid = sx.sx_server_submit(s, **mid_r)
    sids = [sx.sx_server_submit(s, **r) for r in shorts]
    _check_all(s, sids + [mid, lid], shorts + [mid_r, long_r], "short and long")
    st = sx.sx_server_stats_get(s)
    # the first step takes the shorts and the mid request whole (SRPT), the long one in ranges
    assert st["fused"] == len(shorts) + (0 if split else 1), st
    assert 1 <= st["early_done"] <= st["fused"], st
    sx.sx_server_destroy(s)


@pytest.mark.parametrize("split", [0, 1])
def test_single_request_in_one_or_two_steps(target, split):
    """One FP64 triad request of 2^24 elements (640 MiB of work) with a 2 GiB step budget: by
    default one construct-then-operate step (its inputs computed in registers, stored, and the
    operation applied to them), with split_phases a construction step and then an operation
    step (the request is over a quarter of the budget).  Both leave the oracle's inputs and
    result."""
    r = dict(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=1 << 24, q=3.0, seed_x=11, seed_y=12, lo=-1.0, hi=1.0)
    s = sx.sx_server_create(target, budget_bytes=1 << 30, chunk_bytes=(2 << 30) - 1, split_phases=split)
    rid = sx.sx_server_submit(s, **r)
    _check_all(s, [rid], [r], f"split_phases={split}")
    st = sx.sx_server_stats_get(s)
    assert st["steps"] == (2 if split else 1) and st["fused"] == (0 if split else 1), st
    assert st["bytes_moved"] == 40 * (1 << 24)
    sx.sx_server_destroy(s)


def test_fused_requests_with_a_general_range(target):
    """A construct-then-operate piece builds its inputs over any [lo, hi) in both types, in one
    tile or in several (16 KiB tiles: a 4097-element FP64 triad is 11 tiles)."""
    reqs = [dict(op=op, dtype=dt, n=n, q=2.5, seed_x=7 + n, seed_y=8 + n, lo=-3.0, hi=5.5)
            for op in (sx.SX_OP_SCALE, sx.SX_OP_TRIAD) for dt in (sx.SX_F64, sx.SX_F32)
            for n in (1, 63, 4097)]
    for tile in (0, 16384):
        s = sx.sx_server_create(target, budget_bytes=1 << 30, chunk_bytes=1 << 20, tile_bytes=tile)
        ids = [sx.sx_server_submit(s, **r) for r in reqs]
        _check_all(s, ids, reqs, f"tile {tile}")
        assert sx.sx_server_stats_get(s)["fused"] == len(reqs)
        sx.sx_server_destroy(s)


@pytest.mark.parametrize("split", [0, 1])
def test_ranged_pieces_with_a_general_range(target, split):
    """Long requests over a general input range [lo, hi), both types and all four ops, cut into
    many pieces (1 MiB steps, 16 KiB tiles) that share steps with each other: every piece builds
    its range of the inputs at its generator indices and applies the operation to it (or, with
    split_phases, in two phases).  Inputs and results are the oracle's bit for bit."""
    reqs = [dict(op=op, dtype=dt, n=n, q=q, seed_x=31 + 7 * k, seed_y=32 + 7 * k, lo=-3.0, hi=5.5)
            for k, (op, dt, n, q) in enumerate(
                (op, dt, n, q) for op in (sx.SX_OP_COPY, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_TRIAD)
                for dt in (sx.SX_F64, sx.SX_F32) for n, q in ((100003, 3.0), (262147, -0.7)))]
    s = sx.sx_server_create(target, budget_bytes=1 << 30, chunk_bytes=1 << 20, tile_bytes=16384,
                            split_phases=split)
    ids = [sx.sx_server_submit(s, **r) for r in reqs]
    _check_all(s, ids, reqs, f"ranged, split_phases={split}")
    st = sx.sx_server_stats_get(s)
    assert st["completed"] == len(reqs) and st["steps"] > len(reqs) // 2, st
    sx.sx_server_destroy(s)


def test_completion_words_are_recycled(target):
    """More whole-request pieces over a server's life than it has completion words (4096): every
    word goes back to the pool when its request completes, so 6000 short requests (submitted in
    waves, so that many are in flight at once) all complete, each with the oracle's result on a
    sample, and the pool never runs dry for good."""
    s = sx.sx_server_create(target, budget_bytes=1 << 30, chunk_bytes=1 << 20)
    total, wave = 6000, 750
    reqs = [dict(op=[sx.SX_OP_COPY, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_TRIAD][k % 4],
                 dtype=sx.SX_F64 if k % 2 else sx.SX_F32, n=64 + (k * 37) % 900, q=-1.5,
                 seed_x=5000 + k, seed_y=9000 + k, lo=-1.0, hi=1.0) for k in range(total)]
    for first in range(0, total, wave):
        batch = reqs[first:first + wave]
        ids = [sx.sx_server_submit(s, **r) for r in batch]
        checked = [(rid, r) for k, (rid, r) in enumerate(zip(ids, batch)) if k % 50 == 0]
        _check_all(s, [i for i, _ in checked], [r for _, r in checked], f"wave {first // wave}")
        for k, rid in enumerate(ids):
            if k % 50:
                st = sx.sx_server_wait(s, rid, 60000)
                assert st["state"] == sx.SX_REQ_DONE, st
                sx.sx_server_release(s, rid)
    st = sx.sx_server_stats_get(s)
    assert st["completed"] == total and st["fused"] == total, st
    assert 0 < st["early_done"] <= total and st["arena_used"] == 0, st
    sx.sx_server_destroy(s)


def test_replayed_poisson_stream(target):
    reqs = _requests(150, seed=5)
    arr = si.poisson_requests(5, 150, rate_per_s=20000.0)
    t = [a["t"] for a in arr]
    s = sx.sx_server_create(target, budget_bytes=512 << 20, chunk_bytes=4 << 20)
    ids = sx.sx_server_replay(s, [sx.sx_request(**r) for r in reqs], t)
    _check_all(s, ids, reqs, "replay")
    sx.sx_server_destroy(s)


def test_admission_waits_for_memory_and_rejects_oversize(target):
    # each request holds 3 arrays of 1 MiB (F64, n = 2^17): at most 2 fit in an 8 MiB arena
    n = 1 << 17
    s = sx.sx_server_create(target, budget_bytes=8 << 20, chunk_bytes=1 << 20)
    reqs = [dict(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=n, q=3.0, seed_x=10 + k, seed_y=20 + k,
                 lo=-1.0, hi=1.0, flags=sx.SX_REQ_AUTO_RELEASE) for k in range(10)]
    ids = [sx.sx_server_submit(s, **r) for r in reqs]
    big = sx.sx_server_submit(s, op=sx.SX_OP_COPY, dtype=sx.SX_F64, n=1 << 20)  # 16 MiB > arena
    st = sx.sx_server_poll(s, big)
    assert st["state"] == sx.SX_REQ_REJECTED and st["status"] == sx.SX_ERR_OOM
    for rid in ids:
        st = sx.sx_server_wait(s, rid, 60000)
        assert st["state"] == sx.SX_REQ_DONE and st["out"] is None  # auto-released
    stats = sx.sx_server_stats_get(s)
    assert stats["completed"] == 10 and stats["rejected"] == 1
    assert stats["arena_peak"] <= 8 << 20 and stats["arena_used"] == 0
    sx.sx_server_destroy(s)


def test_short_requests_overtake_a_long_one(target):
    """Continuous batching: short requests that arrive while a long one runs finish before it;
    with the per-call FIFO they finish after it.  Arrivals are replayed by the library."""
    long_req = sx.sx_request(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=1 << 28, q=3.0, seed_x=1,
                             seed_y=2, lo=-1.0, hi=1.0, flags=sx.SX_REQ_AUTO_RELEASE)
    short_req = sx.sx_request(op=sx.SX_OP_ADD, dtype=sx.SX_F32, n=1 << 12, q=3.0, seed_x=3,
                              seed_y=4, lo=-1.0, hi=1.0, flags=sx.SX_REQ_AUTO_RELEASE)
    times = [0.0] + [2e-4 + 5e-5 * k for k in range(8)]  # shorts while the long one runs
    order = {}
    for mode in (sx.SX_SERVE_CONTINUOUS, sx.SX_SERVE_FIFO):
        s = sx.sx_server_create(target, budget_bytes=8 << 30, mode=mode, chunk_bytes=64 << 20)
        ids = sx.sx_server_replay(s, [long_req] + [short_req] * 8, times)
        done = [sx.sx_server_wait(s, r, 60000)["t_done"] for r in ids]
        order[mode] = (sum(t < done[0] for t in done[1:]), [round((t - done[0]) * 1e3, 3) for t in done[1:]])
        sx.sx_server_destroy(s)
    assert order[sx.SX_SERVE_CONTINUOUS][0] == 8, order
    assert order[sx.SX_SERVE_FIFO][0] == 0, order


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("backlog", [0, -1])
def test_backlog_steps_only_while_requests_wait(target, backlog, split):
    """Two slots for six requests, so that four wait for admission: with the default backlog the
    server keeps up to steps_in_flight + 2 steps on the GPU while they wait (each step here runs
    ~45 us, much longer than planning one), with backlog_steps = -1 at most steps_in_flight; the
    results equal the oracle's either way.  With split phases the operation pieces wait on the
    device for inputs built by steps still in flight, up to three steps back."""
    reqs = [dict(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=1 << 24, q=3.0, seed_x=40 + k, seed_y=50 + k,
                 lo=-1.0, hi=1.0) for k in range(6)]
    s = sx.sx_server_create(target, budget_bytes=2 << 30, max_active=2, chunk_bytes=256 << 20,
                            steps_in_flight=2, backlog_steps=backlog, split_phases=split)
    ids = [sx.sx_server_submit(s, **r) for r in reqs]
    _check_all(s, ids, reqs, f"backlog {backlog} split {split}")
    st = sx.sx_server_stats_get(s)
    sx.sx_server_destroy(s)
    if backlog == -1:
        assert st["steps_in_flight_peak"] <= 2 and st["backlog_launches"] == 0, st
    else:
        assert 3 <= st["steps_in_flight_peak"] <= 4 and st["backlog_launches"] >= 1, st


def test_a_lone_request_gets_no_backlog_steps(target):
    """Nothing waits for admission: however long the request, at most steps_in_flight steps."""
    r = dict(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=1 << 24, q=3.0, seed_x=60, seed_y=61, lo=-1.0, hi=1.0)
    s = sx.sx_server_create(target, budget_bytes=1 << 30, chunk_bytes=64 << 20)
    ids = [sx.sx_server_submit(s, **r)]
    _check_all(s, ids, [r], "lone request")
    st = sx.sx_server_stats_get(s)
    sx.sx_server_destroy(s)
    assert st["steps"] >= 8 and st["steps_in_flight_peak"] <= 2 and st["backlog_launches"] == 0, st


def test_bad_calls(target):
    with pytest.raises(sx.SxError):
        sx.sx_server_create(target, budget_bytes=0)
    for kw in (dict(steps_in_flight=8, backlog_steps=1), dict(backlog_steps=-2), dict(steps_in_flight=6, backlog_steps=3)):
        with pytest.raises(sx.SxError) as ei:
            sx.sx_server_create(target, budget_bytes=1 << 20, **kw)
        assert ei.value.status == sx.SX_ERR_INVALID, kw
    s = sx.sx_server_create(target, budget_bytes=1 << 20, steps_in_flight=8)  # no room left: no backlog
    sx.sx_server_destroy(s)
    s = sx.sx_server_create(target, budget_bytes=1 << 20)
    with pytest.raises(sx.SxError) as ei:
        sx.sx_server_submit(s, op=7, dtype=sx.SX_F64, n=10)
    assert ei.value.status == sx.SX_ERR_INVALID
    with pytest.raises(sx.SxError) as ei:
        sx.sx_server_release(s, 12345)
    assert ei.value.status == sx.SX_ERR_INVALID
    with pytest.raises(sx.SxError) as ei:
        sx.sx_server_wait(s, 999, 10)
    sx.sx_server_destroy(s)


@pytest.mark.parametrize("policy", [sx.SX_SERVE_POLICY_SRPT, sx.SX_SERVE_POLICY_FAIR,
                                    sx.SX_SERVE_POLICY_SHORT_FIRST])
@pytest.mark.parametrize("serialize", [0, 1])
def test_policies_and_step_overlap(target, policy, serialize):
    """Both sharing policies, with consecutive steps overlapping (operation pieces whose inputs
    were built in a step still running wait for it) and strictly serialized."""
    reqs = _requests(160, seed=6, lo_exp=6, hi_exp=20)
    s = sx.sx_server_create(target, budget_bytes=512 << 20, chunk_bytes=2 << 20, tile_bytes=16384,
                            steps_in_flight=4, policy=policy, serialize_steps=serialize)
    ids = [sx.sx_server_submit(s, **r) for r in reqs]
    _check_all(s, ids, reqs, f"policy {policy} serialize {serialize}")
    assert sx.sx_server_stats_get(s)["steps"] > 10
    sx.sx_server_destroy(s)


def test_served_full_size_requests(target):
    """Requests of the served workload's upper sizes (up to 2^28 elements, 6 GiB of arrays each)
    in a 64 GB arena, mixed with short ones, checked on sampled elements and whole short
    outputs."""
    import torch  # noqa: F401  (device already initialised by the target)
    reqs = []
    for k, n in enumerate([1 << 28, 3 << 25, 4096, 1 << 27, 12345, (1 << 26) + 3, 777, 1 << 20]):
        reqs.append(dict(op=[sx.SX_OP_TRIAD, sx.SX_OP_SCALE, sx.SX_OP_ADD, sx.SX_OP_COPY][k % 4],
                         dtype=sx.SX_F64 if k % 3 else sx.SX_F32, n=n, q=3.0,
                         seed_x=int(si.word_scalar(77, 2 * k)), seed_y=int(si.word_scalar(77, 2 * k + 1)),
                         lo=-1.0, hi=1.0))
    s = sx.sx_server_create(target, budget_bytes=64 << 30)
    ids = [sx.sx_server_submit(s, **r) for r in reqs]
    rng = np.random.default_rng(4)
    for rid, r in zip(ids, reqs):
        st = sx.sx_server_wait(s, rid, 120000)
        assert st["state"] == sx.SX_REQ_DONE
        n, dt = r["n"], NP[r["dtype"]]
        if n <= (1 << 20):
            x, y, want = _expected(r)
            assert np.array_equal(_read(s, rid, 2, r).view(np.uint8), want.view(np.uint8))
        else:
            idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 4096)]))
            es = np.dtype(dt).itemsize
            out = np.empty(idx.size, dt)
            for m, i in enumerate(idx):  # single-element reads from the resident result
                wrap = sx.sx_array_wrap(target, r["dtype"], st["out"] + es * int(i), 1)
                sx.sx_copy_d2h(out[m:m + 1].ctypes.data, wrap, 1)
                sx.sx_free(wrap)
            xs = si.uniform_at(r["seed_x"], idx.astype(np.uint64), dt)
            ys = si.uniform_at(r["seed_y"], idx.astype(np.uint64), dt)
            want = oracle.apply(OPN[r["op"]], xs, ys, r["q"])
            assert np.array_equal(out.view(np.uint8), want.view(np.uint8)), (rid, r["op"], n)
        sx.sx_server_release(s, rid)
    sx.sx_server_destroy(s)


def test_release_during_a_read_waits_for_the_read(target):
    """A request is released (and a second request that can only fit in the same memory is
    submitted) while another thread is still copying the first one's output to the host: the
    copy sees the first result intact, the second request is admitted only after the copy, and
    a read after the release is refused."""
    import threading
    import time
    n = 1 << 25
    a = dict(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=n, q=3.0, seed_x=11, seed_y=12, lo=-1.0, hi=1.0)
    b = dict(a, seed_x=21, seed_y=22)
    s = sx.sx_server_create(target, budget_bytes=3 * 8 * n + (1 << 20))
    try:
        ra = sx.sx_server_submit(s, **a)
        assert sx.sx_server_wait(s, ra, 60000)["state"] == sx.SX_REQ_DONE
        got = np.empty(n, np.float64)
        reads = []
        th = threading.Thread(target=lambda: reads.append(
            sx.sx_server_read(s, ra, 2, got.ctypes.data, n)))
        th.start()
        time.sleep(0.002)
        sx.sx_server_release(s, ra)
        rb = sx.sx_server_submit(s, **b)
        th.join()
        with pytest.raises(sx.SxError) as ei:
            sx.sx_server_read(s, ra, 2, got.ctypes.data, 1)
        assert ei.value.status == sx.SX_ERR_STATE
        assert np.array_equal(got.view(np.uint64), _expected(a)[2].view(np.uint64))
        st = sx.sx_server_wait(s, rb, 60000)
        assert st["state"] == sx.SX_REQ_DONE
        assert np.array_equal(_read(s, rb, 2, b).view(np.uint64), _expected(b)[2].view(np.uint64))
        sx.sx_server_release(s, rb)
    finally:
        sx.sx_server_destroy(s)


@pytest.mark.parametrize("mode", [sx.SX_SERVE_CONTINUOUS, sx.SX_SERVE_FIFO])
def test_requests_with_special_scalars(target, mode):
    """FP64 and FP32 scale/triad requests whose scalar is infinite, zero, subnormal, huge or has
    a long significand: results equal the oracle (NaN positions as NaN) in both modes."""
    qs = [float("inf"), -0.0, 5e-324, 2.0 ** -1022, 1.7976931348623157e308, 1.0 / 3.0, -7.5]
    reqs = []
    for k, q in enumerate(qs):
        for op in (sx.SX_OP_SCALE, sx.SX_OP_TRIAD):
            for dt in (sx.SX_F64, sx.SX_F32):
                reqs.append(dict(op=op, dtype=dt, n=1000 + 37 * k, q=q, seed_x=500 + k, seed_y=600 + k,
                                 lo=-1.0, hi=1.0))
    s = sx.sx_server_create(target, budget_bytes=1 << 28, mode=mode)
    try:
        ids = [sx.sx_server_submit(s, **r) for r in reqs]
        for rid, r in zip(ids, reqs):
            assert sx.sx_server_wait(s, rid, 60000)["state"] == sx.SX_REQ_DONE
            got = _read(s, rid, 2, r)
            want = _expected(r)[2]
            ok = ~np.isnan(want)
            assert np.array_equal(got[ok].view(np.uint8), want[ok].view(np.uint8)), (r["q"], OPN[r["op"]])
            assert np.array_equal(np.isnan(got), np.isnan(want)), (r["q"], OPN[r["op"]])
            sx.sx_server_release(s, rid)
    finally:
        sx.sx_server_destroy(s)


@pytest.mark.parametrize("mode", [sx.SX_SERVE_CONTINUOUS, sx.SX_SERVE_FIFO])
def test_cancel_queued_active_and_finished(target, mode):
    """A queued request leaves the queue; an active one launches no further work and is
    CANCELLED once the work already in flight completes, its memory freed for the next request
    (which computes correctly in it); a finished request cannot be cancelled."""
    n = 1 << 26
    big = dict(op=sx.SX_OP_TRIAD, dtype=sx.SX_F64, n=n, q=3.0, seed_x=1, seed_y=2, lo=-1.0, hi=1.0)
    s = sx.sx_server_create(target, budget_bytes=3 * 8 * n + (64 << 20), mode=mode)
    try:
        ra = sx.sx_server_submit(s, **big)
        rb = sx.sx_server_submit(s, **dict(big, seed_x=3))  # waits: the arena holds one such request
        assert sx.sx_server_poll(s, rb)["state"] == sx.SX_REQ_QUEUED
        sx.sx_server_cancel(s, rb)
        assert sx.sx_server_poll(s, rb)["state"] == sx.SX_REQ_CANCELLED
        sx.sx_server_cancel(s, ra)  # active (or, if very fast, already cancelled at its last step)
        assert sx.sx_server_wait(s, ra, 60000)["state"] == sx.SX_REQ_CANCELLED
        sx.sx_server_release(s, ra)  # nothing to free: a no-op
        with pytest.raises(sx.SxError) as ei:
            sx.sx_server_read(s, ra, 2, np.empty(1).ctypes.data, 1)
        assert ei.value.status == sx.SX_ERR_STATE
        st = sx.sx_server_stats_get(s)
        assert st["cancelled"] == 2 and st["arena_used"] == 0
        d = dict(big, seed_x=5, seed_y=6)
        rd = sx.sx_server_submit(s, **d)
        assert sx.sx_server_wait(s, rd, 60000)["state"] == sx.SX_REQ_DONE
        assert np.array_equal(_read(s, rd, 2, d).view(np.uint64), _expected(d)[2].view(np.uint64))
        with pytest.raises(sx.SxError) as ei:
            sx.sx_server_cancel(s, rd)
        assert ei.value.status == sx.SX_ERR_STATE
        sx.sx_server_release(s, rd)
        with pytest.raises(sx.SxError) as ei:
            sx.sx_server_cancel(s, 10 ** 9)
        assert ei.value.status == sx.SX_ERR_INVALID
    finally:
        sx.sx_server_destroy(s)


@pytest.mark.parametrize("mode", [sx.SX_SERVE_CONTINUOUS, sx.SX_SERVE_FIFO])
def test_concurrent_clients(target, mode):
    """Eight client threads each submit, wait for, read, check and release (or cancel) their own
    stream of requests against one server: every completed result equals the oracle's, every
    request ends DONE or CANCELLED, and the arena is empty at the end."""
    import threading
    threads, per_thread = 8, 24
    s = sx.sx_server_create(target, budget_bytes=1 << 28, mode=mode)
    errors, cancelled = [], [0]
    lock = threading.Lock()

    def client(k):
        try:
            reqs = _requests(per_thread, 900 + k, lo_exp=4, hi_exp=16)
            rng = np.random.default_rng(k)
            for i, r in enumerate(reqs):
                rid = sx.sx_server_submit(s, **r)
                if rng.random() < 0.2:
                    try:
                        sx.sx_server_cancel(s, rid)
                    except sx.SxError as e:  # it may have finished already
                        assert e.status == sx.SX_ERR_STATE
                st = sx.sx_server_wait(s, rid, 60000)
                if st["state"] == sx.SX_REQ_CANCELLED:
                    with lock:
                        cancelled[0] += 1
                    continue
                assert st["state"] == sx.SX_REQ_DONE, st
                want = _expected(r)[2]
                got = _read(s, rid, 2, r)
                assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (k, i)
                sx.sx_server_release(s, rid)
        except Exception as e:  # reported by the main thread
            errors.append((k, repr(e)))

    ts = [threading.Thread(target=client, args=(k,)) for k in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    try:
        assert not errors, errors[:3]
        st = sx.sx_server_stats_get(s)
        assert st["submitted"] == threads * per_thread
        assert st["completed"] + st["cancelled"] == threads * per_thread
        assert st["cancelled"] == cancelled[0]
        assert st["arena_used"] == 0
    finally:
        sx.sx_server_destroy(s)
