"""Helpers for the GPU tests: host<->device staging through the C ABI and bitwise comparison."""
import numpy as np

import paper_2206_06302_b300 as sx

NP = {sx.SX_F32: np.float32, sx.SX_F64: np.float64, sx.SX_U8: np.uint8}
CODE = {np.dtype(np.float32): sx.SX_F32, np.dtype(np.float64): sx.SX_F64,
        np.dtype(np.uint8): sx.SX_U8}


def to_device(t, host: np.ndarray):
    host = np.ascontiguousarray(host)
    a = sx.sx_alloc(t, CODE[host.dtype], host.size)
    if host.size:
        sx.sx_copy_h2d(a, host.ctypes.data, host.size)
    return a


def empty(t, dtype, n):
    return sx.sx_alloc(t, CODE[np.dtype(dtype)], n)


def to_host(a) -> np.ndarray:
    _, n, dt = sx.sx_array_data(a)
    out = np.empty(n, NP[dt])
    if n:
        sx.sx_copy_d2h(out.ctypes.data, a, n)
    return out


def bits(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    return a.view({8: np.uint64, 4: np.uint32, 1: np.uint8}[a.dtype.itemsize])


def assert_bitwise(got: np.ndarray, want: np.ndarray, what=""):
    assert got.dtype == want.dtype and got.shape == want.shape, what
    gb, wb = bits(got), bits(want)
    if not np.array_equal(gb, wb):
        bad = np.flatnonzero(gb != wb)
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} of {got.size} elements differ; first at {i}: "
                             f"got {got[i]!r} ({gb[i]:#x}) want {want[i]!r} ({wb[i]:#x})")
