"""Thin ctypes binding of libsx (``include/sx.h``): the same names, argument marshalling only.

Every STREAM step runs in the CUDA library; this module converts Python values to C
arguments, turns non-zero status codes into :class:`SxError`, and returns out-parameters.
If ``libsx.so`` is missing the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsx.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libsx.so not found at {LIB_PATH}: build it with "
        "`python paper_2206_06302_b300/build.py` (there is no CPU fallback)")
lib = C.CDLL(LIB_PATH)

# ---- constants (mirror sx.h) -----------------------------------------------------------------
SX_OK, SX_ERR_INVALID, SX_ERR_OOM, SX_ERR_DTYPE, SX_ERR_OVERLAP = 0, 1, 2, 3, 4
SX_ERR_TIMEOUT, SX_ERR_CUDA, SX_ERR_NOT_READY, SX_ERR_DEVICE, SX_ERR_STATE = 5, 6, 7, 8, 9
SX_F32, SX_F64, SX_U8 = 1, 2, 3
SX_OP_COPY, SX_OP_SCALE, SX_OP_ADD, SX_OP_TRIAD, SX_OP_SEED = 0, 1, 2, 3, 4
SX_PAR, SX_PAR_TASK = 1, 2
SX_VARIANT_AUTO, SX_VARIANT_VECTOR, SX_VARIANT_BULK, SX_VARIANT_TMA, SX_VARIANT_TMA_TENSOR = 0, 1, 2, 3, 4
SX_FN_TO_UPPER, SX_FN_TO_LOWER = 1, 2
SX_SERVE_CONTINUOUS, SX_SERVE_FIFO = 0, 1
SX_SERVE_POLICY_SRPT, SX_SERVE_POLICY_FAIR, SX_SERVE_POLICY_SHORT_FIRST = 0, 1, 2
SX_REQ_QUEUED, SX_REQ_ACTIVE, SX_REQ_DONE, SX_REQ_REJECTED, SX_REQ_RELEASED, SX_REQ_CANCELLED = 0, 1, 2, 3, 4, 5
SX_REQ_AUTO_RELEASE = 1
SX_NOALLOC_MAX_ITEMS, SX_NOALLOC_MAX_TILES, SX_NOALLOC_SCRATCH_BYTES = 4096, 65536, 950272

OPS = {"copy": SX_OP_COPY, "scale": SX_OP_SCALE, "add": SX_OP_ADD, "triad": SX_OP_TRIAD,
       "seed": SX_OP_SEED}
DTYPES = {"f32": SX_F32, "f64": SX_F64, "u8": SX_U8}


class SxError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        super().__init__(f"{func}: {lib.sx_status_string(status).decode()}: {msg}")


# ---- structures --------------------------------------------------------------------------------
class sx_launch_cfg(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("variant", "threads", "blocks_per_sm", "vec_bytes",
                                         "unroll", "cache_hint", "tile_bytes", "stages",
                                         "fp64_mul", "reserved")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class sx_target_info(C.Structure):
    _fields_ = [("device", C.c_int32), ("sm_count", C.c_int32), ("cc_major", C.c_int32),
                ("cc_minor", C.c_int32), ("l2_bytes", C.c_int64), ("hbm_total", C.c_int64),
                ("hbm_free", C.c_int64), ("budget", C.c_int64), ("used", C.c_int64),
                ("max_smem_block", C.c_int32), ("sm_clock_khz", C.c_int32),
                ("name", C.c_char * 128)]


class sx_batch_item(C.Structure):
    _fields_ = [("op", C.c_int32), ("dtype", C.c_int32), ("n", C.c_uint64),
                ("x", C.c_void_p), ("y", C.c_void_p), ("out", C.c_void_p),
                ("q", C.c_double), ("q2", C.c_double), ("seed", C.c_uint64),
                ("index_base", C.c_uint64)]


class sx_batch_cfg(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("chunk_bytes", "threads", "blocks_per_sm", "vec_bytes")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class sx_server_cfg(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("mode", C.c_int32), ("max_active", C.c_int32),
                ("chunk_bytes", C.c_int32), ("steps_in_flight", C.c_int32),
                ("threads", C.c_int32), ("blocks_per_sm", C.c_int32), ("vec_bytes", C.c_int32),
                ("tile_bytes", C.c_int32), ("policy", C.c_int32), ("serialize_steps", C.c_int32),
                ("split_phases", C.c_int32), ("backlog_steps", C.c_int32)]


class sx_request(C.Structure):
    _fields_ = [("op", C.c_int32), ("dtype", C.c_int32), ("n", C.c_uint64), ("q", C.c_double),
                ("seed_x", C.c_uint64), ("seed_y", C.c_uint64), ("lo", C.c_double),
                ("hi", C.c_double), ("flags", C.c_uint32), ("reserved", C.c_uint32)]


class sx_request_status(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("x", C.c_void_p),
                ("y", C.c_void_p), ("out", C.c_void_p)]


class sx_server_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "admitted", "completed", "rejected",
                                          "steps", "launches", "bytes_moved", "arena_used",
                                          "arena_peak", "arena_bytes")] + [(n, C.c_double) for n in (
                                              "busy_seconds", "host_step_seconds", "host_admit_seconds")] + [
        ("cancelled", C.c_uint64), ("fused", C.c_uint64), ("early_done", C.c_uint64),
        ("steps_in_flight_peak", C.c_uint64), ("backlog_launches", C.c_uint64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


# ---- prototypes ----------------------------------------------------------------------------------
P, I, U64, SZ, D = C.c_void_p, C.c_int, C.c_uint64, C.c_size_t, C.c_double
PP = C.POINTER(C.c_void_p)

_PROTOS = {
    "sx_target_count": [C.POINTER(C.c_int)],
    "sx_target_create": [I, PP],
    "sx_target_create_ext": [I, P, SZ, PP],
    "sx_target_destroy": [P],
    "sx_target_info_get": [P, C.POINTER(sx_target_info)],
    "sx_target_stream": [P, PP],
    "sx_target_synchronize": [P],
    "sx_target_selftest": [P, C.c_int64],
    "sx_alloc": [P, I, SZ, PP],
    "sx_array_wrap": [P, I, P, SZ, PP],
    "sx_free": [P],
    "sx_array_data": [P, PP, C.POINTER(C.c_size_t), C.POINTER(C.c_int)],
    "sx_array_guard_ok": [P, C.POINTER(C.c_int)],
    "sx_bulk_construct": [P, D],
    "sx_bulk_destroy": [P],
    "sx_seed_uniform": [P, U64, D, D],
    "sx_seed_uniform_at": [P, U64, D, D, U64],
    "sx_block_partition": [U64, I, I, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)],
    "sx_copy_h2d": [P, P, SZ],
    "sx_copy_d2h": [P, P, SZ],
    "sx_copy_h2d_async": [P, P, SZ],
    "sx_copy_d2h_async": [P, P, SZ],
    "sx_executor_create": [P, I, C.POINTER(sx_launch_cfg), PP],
    "sx_executor_destroy": [P],
    "sx_executor_wait": [P],
    "sx_executor_resolve": [P, I, I, SZ, C.POINTER(sx_launch_cfg)],
    "sx_future_wait": [P, C.c_int64],
    "sx_future_test": [P],
    "sx_future_elapsed_ms": [P, C.POINTER(C.c_float)],
    "sx_future_destroy": [P],
    "sx_copy": [P, P, P],
    "sx_transform_scale": [P, P, P, D],
    "sx_transform_add": [P, P, P, P],
    "sx_transform_triad": [P, P, P, P, D],
    "sx_execute": [P, I, P, P, P, D],
    "sx_execute_async": [P, I, P, P, P, D, PP],
    "sx_stream_iter": [P, P, P, P, D, I],
    "sx_stream_fused": [P, P, P, P, D, I],
    "sx_stream_host": [P, P, P, P, P, P, P, D, I],
    "sx_transform_u8": [P, I, P, P],
    "sx_transform_src": [P, C.c_char_p, P, P],
    "sx_batch_create": [P, C.POINTER(sx_batch_item), SZ, C.POINTER(sx_batch_cfg), PP],
    "sx_batch_launch": [P],
    "sx_batch_launch_async": [P, PP],
    "sx_batch_launch_percall": [P, C.POINTER(sx_launch_cfg)],
    "sx_batch_set_record": [P, I],
    "sx_batch_completion_ns": [P, C.POINTER(C.c_uint64), SZ],
    "sx_batch_info": [P, C.POINTER(sx_batch_cfg), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)],
    "sx_batch_destroy": [P],
    "sx_batch_run_noalloc": [P, C.POINTER(sx_batch_item), SZ, C.POINTER(sx_batch_cfg)],
    "sx_tune": [P, I, I, SZ, C.POINTER(sx_launch_cfg), C.POINTER(C.c_float)],
    "sx_tune_pass": [P, I, SZ, C.POINTER(sx_launch_cfg), C.POINTER(C.c_float)],
    "sx_tune_batch": [P, C.POINTER(sx_batch_cfg), C.POINTER(C.c_float)],
    "sx_tune_lookup": [P, I, I, SZ, C.POINTER(sx_launch_cfg)],
    "sx_tune_save": [C.c_char_p],
    "sx_tune_load": [C.c_char_p],
    "sx_tune_clear": [],
    "sx_server_create": [P, C.POINTER(sx_server_cfg), PP],
    "sx_server_submit": [P, C.POINTER(sx_request), C.POINTER(C.c_uint64)],
    "sx_server_replay": [P, C.POINTER(sx_request), C.POINTER(C.c_double), SZ, C.POINTER(C.c_uint64)],
    "sx_server_poll": [P, U64, C.POINTER(sx_request_status)],
    "sx_server_wait": [P, U64, C.c_int64, C.POINTER(sx_request_status)],
    "sx_server_read": [P, U64, I, P, SZ],
    "sx_server_release": [P, U64],
    "sx_server_cancel": [P, U64],
    "sx_server_stats_get": [P, C.POINTER(sx_server_stats)],
    "sx_server_destroy": [P],
}

for _name, _args in _PROTOS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.sx_last_error.restype = C.c_char_p
lib.sx_last_error.argtypes = []
lib.sx_status_string.restype = C.c_char_p
lib.sx_status_string.argtypes = [C.c_int]
lib.sx_version.restype = C.c_int
lib.sx_version.argtypes = []

#: Every function the header declares (for the export test).
EXPORTED = sorted(list(_PROTOS) + ["sx_last_error", "sx_status_string", "sx_version"])


def _check(status: int, func: str, ok=(SX_OK,)) -> int:
    if status not in ok:
        raise SxError(status, func, lib.sx_last_error().decode(errors="replace"))
    return status


def _h(x):
    """Handle value of a wrapper object or a raw pointer."""
    if x is None:
        return None
    return getattr(x, "_as_parameter_", x)


def _cfg(cfg):
    if cfg is None:
        return None
    if isinstance(cfg, sx_launch_cfg):
        return C.byref(cfg)
    c = sx_launch_cfg(**cfg)
    return C.byref(c)


# ---- functions with the header's names -----------------------------------------------------------
def sx_last_error() -> str:
    return lib.sx_last_error().decode(errors="replace")


def sx_status_string(status: int) -> str:
    return lib.sx_status_string(status).decode()


def sx_version() -> int:
    return lib.sx_version()


def sx_target_count() -> int:
    n = C.c_int(0)
    _check(lib.sx_target_count(C.byref(n)), "sx_target_count")
    return n.value


def sx_target_create(device: int = 0):
    h = C.c_void_p()
    _check(lib.sx_target_create(device, C.byref(h)), "sx_target_create")
    return h.value


def sx_target_create_ext(device: int, stream: int | None, budget_bytes: int = 0):
    h = C.c_void_p()
    _check(lib.sx_target_create_ext(device, stream, budget_bytes, C.byref(h)), "sx_target_create_ext")
    return h.value


def sx_target_destroy(t) -> None:
    _check(lib.sx_target_destroy(t), "sx_target_destroy")


def sx_target_info_get(t) -> dict:
    info = sx_target_info()
    _check(lib.sx_target_info_get(t, C.byref(info)), "sx_target_info_get")
    d = {n: getattr(info, n) for n, _ in info._fields_}
    d["name"] = info.name.decode()
    return d


def sx_target_stream(t) -> int:
    s = C.c_void_p()
    _check(lib.sx_target_stream(t, C.byref(s)), "sx_target_stream")
    return s.value or 0


def sx_target_synchronize(t) -> None:
    _check(lib.sx_target_synchronize(t), "sx_target_synchronize")


def sx_target_selftest(t, limit_us: int) -> None:
    _check(lib.sx_target_selftest(t, limit_us), "sx_target_selftest")


def sx_alloc(t, dtype: int, n: int):
    h = C.c_void_p()
    _check(lib.sx_alloc(t, dtype, n, C.byref(h)), "sx_alloc")
    return h.value


def sx_array_wrap(t, dtype: int, device_ptr: int, n: int):
    h = C.c_void_p()
    _check(lib.sx_array_wrap(t, dtype, device_ptr, n, C.byref(h)), "sx_array_wrap")
    return h.value


def sx_free(a) -> None:
    _check(lib.sx_free(a), "sx_free")


def sx_array_data(a):
    p, n, dt = C.c_void_p(), C.c_size_t(), C.c_int()
    _check(lib.sx_array_data(a, C.byref(p), C.byref(n), C.byref(dt)), "sx_array_data")
    return p.value, n.value, dt.value


def sx_array_guard_ok(a) -> bool:
    ok = C.c_int()
    _check(lib.sx_array_guard_ok(a, C.byref(ok)), "sx_array_guard_ok")
    return bool(ok.value)


def sx_bulk_construct(a, value: float) -> None:
    _check(lib.sx_bulk_construct(a, value), "sx_bulk_construct")


def sx_bulk_destroy(a) -> None:
    _check(lib.sx_bulk_destroy(a), "sx_bulk_destroy")


def sx_seed_uniform(a, seed: int, lo: float = -1.0, hi: float = 1.0) -> None:
    _check(lib.sx_seed_uniform(a, seed, lo, hi), "sx_seed_uniform")


def sx_seed_uniform_at(a, seed: int, lo: float = -1.0, hi: float = 1.0, index_base: int = 0) -> None:
    _check(lib.sx_seed_uniform_at(a, seed, lo, hi, index_base), "sx_seed_uniform_at")


def sx_block_partition(n: int, parts: int, part: int) -> tuple[int, int]:
    """(offset, count) of block `part` of n elements divided over `parts` targets."""
    off, cnt = C.c_uint64(), C.c_uint64()
    _check(lib.sx_block_partition(n, parts, part, C.byref(off), C.byref(cnt)), "sx_block_partition")
    return off.value, cnt.value


def sx_copy_h2d(a, host_ptr: int, n: int) -> None:
    _check(lib.sx_copy_h2d(a, host_ptr, n), "sx_copy_h2d")


def sx_copy_d2h(host_ptr: int, a, n: int) -> None:
    _check(lib.sx_copy_d2h(host_ptr, a, n), "sx_copy_d2h")


def sx_copy_h2d_async(a, host_ptr: int, n: int) -> None:
    _check(lib.sx_copy_h2d_async(a, host_ptr, n), "sx_copy_h2d_async")


def sx_copy_d2h_async(host_ptr: int, a, n: int) -> None:
    _check(lib.sx_copy_d2h_async(host_ptr, a, n), "sx_copy_d2h_async")


def sx_executor_create(t, policy: int = SX_PAR, cfg=None):
    h = C.c_void_p()
    _check(lib.sx_executor_create(t, policy, _cfg(cfg), C.byref(h)), "sx_executor_create")
    return h.value


def sx_executor_destroy(e) -> None:
    _check(lib.sx_executor_destroy(e), "sx_executor_destroy")


def sx_executor_wait(e) -> None:
    _check(lib.sx_executor_wait(e), "sx_executor_wait")


def sx_executor_resolve(e, op: int, dtype: int, n: int) -> dict:
    c = sx_launch_cfg()
    _check(lib.sx_executor_resolve(e, op, dtype, n, C.byref(c)), "sx_executor_resolve")
    return c.as_dict()


def sx_future_wait(f, timeout_ms: int = -1) -> None:
    _check(lib.sx_future_wait(f, timeout_ms), "sx_future_wait")


def sx_future_test(f) -> bool:
    return _check(lib.sx_future_test(f), "sx_future_test", ok=(SX_OK, SX_ERR_NOT_READY)) == SX_OK


def sx_future_elapsed_ms(f) -> float:
    ms = C.c_float()
    _check(lib.sx_future_elapsed_ms(f, C.byref(ms)), "sx_future_elapsed_ms")
    return ms.value


def sx_future_destroy(f) -> None:
    _check(lib.sx_future_destroy(f), "sx_future_destroy")


def sx_copy(e, src, dst) -> None:
    _check(lib.sx_copy(e, src, dst), "sx_copy")


def sx_transform_scale(e, x, out, q: float) -> None:
    _check(lib.sx_transform_scale(e, x, out, q), "sx_transform_scale")


def sx_transform_add(e, x, y, out) -> None:
    _check(lib.sx_transform_add(e, x, y, out), "sx_transform_add")


def sx_transform_triad(e, x, y, out, q: float) -> None:
    _check(lib.sx_transform_triad(e, x, y, out, q), "sx_transform_triad")


def sx_execute(e, op: int, x, y, out, q: float = 0.0) -> None:
    _check(lib.sx_execute(e, op, x, y, out, q), "sx_execute")


def sx_execute_async(e, op: int, x, y, out, q: float = 0.0, future: bool = True):
    f = C.c_void_p()
    _check(lib.sx_execute_async(e, op, x, y, out, q, C.byref(f) if future else None),
           "sx_execute_async")
    return f.value if future else None


def sx_stream_iter(e, a, b, c, q: float = 3.0, iters: int = 1) -> None:
    _check(lib.sx_stream_iter(e, a, b, c, q, iters), "sx_stream_iter")


def sx_stream_fused(e, a, b, c, q: float = 3.0, iters: int = 1) -> None:
    _check(lib.sx_stream_fused(e, a, b, c, q, iters), "sx_stream_fused")


def sx_stream_host(e, ha: int, hb: int, hc: int, a, b, c, q: float = 3.0, iters: int = 1) -> None:
    _check(lib.sx_stream_host(e, ha, hb, hc, a, b, c, q, iters), "sx_stream_host")


def sx_transform_u8(e, fn: int, x, out) -> None:
    _check(lib.sx_transform_u8(e, fn, x, out), "sx_transform_u8")


def sx_transform_src(e, src: str, x, out) -> None:
    """out[i] = sx_fn(x[i]) with sx_fn defined by the CUDA C++ source `src` (compiled at run time)."""
    _check(lib.sx_transform_src(e, src.encode(), x, out), "sx_transform_src")


def sx_batch_create(t, items, cfg=None):
    arr = (sx_batch_item * len(items))(*items)
    h = C.c_void_p()
    c = None
    if cfg is not None:
        c = C.byref(cfg if isinstance(cfg, sx_batch_cfg) else sx_batch_cfg(**cfg))
    _check(lib.sx_batch_create(t, arr, len(items), c, C.byref(h)), "sx_batch_create")
    return h.value


def sx_batch_launch(b) -> None:
    _check(lib.sx_batch_launch(b), "sx_batch_launch")


def sx_batch_launch_async(b) -> int:
    """bulk_async_execute: launch the batch and return a future (destroy it when done)."""
    f = C.c_void_p()
    _check(lib.sx_batch_launch_async(b, C.byref(f)), "sx_batch_launch_async")
    return f.value


def sx_batch_launch_percall(b, cfg=None) -> None:
    _check(lib.sx_batch_launch_percall(b, _cfg(cfg)), "sx_batch_launch_percall")


def sx_batch_set_record(b, record: bool) -> None:
    _check(lib.sx_batch_set_record(b, int(record)), "sx_batch_set_record")


def sx_batch_completion_ns(b, count: int):
    buf = (C.c_uint64 * count)()
    _check(lib.sx_batch_completion_ns(b, buf, count), "sx_batch_completion_ns")
    return list(buf)


def sx_batch_info(b):
    c, tiles, nbytes = sx_batch_cfg(), C.c_uint64(), C.c_uint64()
    _check(lib.sx_batch_info(b, C.byref(c), C.byref(tiles), C.byref(nbytes)), "sx_batch_info")
    return c.as_dict(), tiles.value, nbytes.value


def sx_batch_destroy(b) -> None:
    _check(lib.sx_batch_destroy(b), "sx_batch_destroy")


def sx_batch_run_noalloc(stream: int | None, items, cfg=None) -> None:
    """Run `items` once on `stream` without allocating device memory (see sx.h)."""
    arr = (sx_batch_item * max(1, len(items)))(*items)
    c = None
    if cfg is not None:
        c = C.byref(cfg if isinstance(cfg, sx_batch_cfg) else sx_batch_cfg(**cfg))
    _check(lib.sx_batch_run_noalloc(stream, arr, len(items), c), "sx_batch_run_noalloc")


def sx_tune(t, op: int, dtype: int, n: int):
    c, gbs = sx_launch_cfg(), C.c_float()
    _check(lib.sx_tune(t, op, dtype, n, C.byref(c), C.byref(gbs)), "sx_tune")
    return c.as_dict(), gbs.value


def sx_tune_pass(t, dtype: int, n: int):
    """The four pass kernels' shapes (copy, scale, add, triad) and the pass's GB/s."""
    c, gbs = (sx_launch_cfg * 4)(), C.c_float()
    _check(lib.sx_tune_pass(t, dtype, n, c, C.byref(gbs)), "sx_tune_pass")
    return [x.as_dict() for x in c], gbs.value


def sx_tune_batch(b):
    c, ms = sx_batch_cfg(), C.c_float()
    _check(lib.sx_tune_batch(b, C.byref(c), C.byref(ms)), "sx_tune_batch")
    return c.as_dict(), ms.value


def sx_tune_lookup(t, op: int, dtype: int, n: int):
    c = sx_launch_cfg()
    st = _check(lib.sx_tune_lookup(t, op, dtype, n, C.byref(c)), "sx_tune_lookup",
                ok=(SX_OK, SX_ERR_NOT_READY))
    return c.as_dict() if st == SX_OK else None


def sx_tune_save(path: str) -> None:
    _check(lib.sx_tune_save(path.encode()), "sx_tune_save")


def sx_tune_load(path: str) -> None:
    _check(lib.sx_tune_load(path.encode()), "sx_tune_load")


def sx_tune_clear() -> None:
    _check(lib.sx_tune_clear(), "sx_tune_clear")


def sx_server_create(t, **cfg):
    c = sx_server_cfg(**cfg)
    h = C.c_void_p()
    _check(lib.sx_server_create(t, C.byref(c), C.byref(h)), "sx_server_create")
    return h.value


def sx_server_submit(s, op: int, dtype: int, n: int, q: float = 3.0, seed_x: int = 1,
                     seed_y: int = 2, lo: float = -1.0, hi: float = 1.0, flags: int = 0) -> int:
    r = sx_request(op=op, dtype=dtype, n=n, q=q, seed_x=seed_x, seed_y=seed_y, lo=lo, hi=hi,
                   flags=flags)
    rid = C.c_uint64()
    _check(lib.sx_server_submit(s, C.byref(r), C.byref(rid)), "sx_server_submit")
    return rid.value


def sx_server_replay(s, requests, t_arrival) -> list:
    """Submit `requests` (sx_request or dicts) at `t_arrival` seconds from now, from a library
    thread; returns their ids at once."""
    k = len(requests)
    reqs = (sx_request * k)(*[r if isinstance(r, sx_request) else sx_request(**r) for r in requests])
    ts = (C.c_double * k)(*t_arrival)
    ids = (C.c_uint64 * k)()
    _check(lib.sx_server_replay(s, reqs, ts, k, ids), "sx_server_replay")
    return list(ids)


def _status_dict(st: sx_request_status) -> dict:
    return {n: getattr(st, n) for n, _ in st._fields_}


def sx_server_poll(s, rid: int) -> dict:
    st = sx_request_status()
    _check(lib.sx_server_poll(s, rid, C.byref(st)), "sx_server_poll")
    return _status_dict(st)


def sx_server_wait(s, rid: int, timeout_ms: int = -1) -> dict:
    st = sx_request_status()
    _check(lib.sx_server_wait(s, rid, timeout_ms, C.byref(st)), "sx_server_wait")
    return _status_dict(st)


def sx_server_read(s, rid: int, which: int, host_ptr: int, n: int) -> None:
    _check(lib.sx_server_read(s, rid, which, host_ptr, n), "sx_server_read")


def sx_server_release(s, rid: int) -> None:
    _check(lib.sx_server_release(s, rid), "sx_server_release")


def sx_server_cancel(s, rid: int) -> None:
    _check(lib.sx_server_cancel(s, rid), "sx_server_cancel")


def sx_server_stats_get(s) -> dict:
    st = sx_server_stats()
    _check(lib.sx_server_stats_get(s, C.byref(st)), "sx_server_stats_get")
    return st.as_dict()


def sx_server_destroy(s) -> None:
    _check(lib.sx_server_destroy(s), "sx_server_destroy")
