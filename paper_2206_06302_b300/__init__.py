"""STREAM over execution targets on one B300 GPU (Heller et al., "Closing the Performance Gap
with Modern C++": targets, placing allocators, executors, and STREAM as parallel algorithms).

The compute path is ``libsx.so`` (CUDA for sm_103a, C ABI in ``include/sx.h``); :mod:`.sx` is its
ctypes binding with the header's names.  This module adds two torch conveniences: a target
that enqueues on a torch stream, and wrapping a CUDA tensor's storage as a borrowed array.
Importing fails loudly if the library has not been built.

On import the tuner table shipped with the package (``tune_b300.json``: launch shapes measured
on B300 for the four kernels, both types, array sizes 2^16..2^29) is loaded, so executors that
leave the variant at AUTO use it; entries for other devices are ignored by the lookup.
"""
from __future__ import annotations

import os

from . import sx
from .sx import *  # noqa: F401,F403  (the header's names)

__all__ = [n for n in dir(sx) if n.startswith(("sx_", "SX_"))] + [
    "sx", "SxError", "target_on_torch_stream", "wrap_tensor", "dtype_of", "SHIPPED_TUNE_TABLE",
    "load_shipped_tune_table"]

SHIPPED_TUNE_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_b300.json")


def load_shipped_tune_table() -> bool:
    """Load the shipped tuner table into the library's table (True if it exists)."""
    if os.path.exists(SHIPPED_TUNE_TABLE):
        sx.sx_tune_load(SHIPPED_TUNE_TABLE)
        return True
    return False


load_shipped_tune_table()


def dtype_of(tensor) -> int:
    import torch
    m = {torch.float32: sx.SX_F32, torch.float64: sx.SX_F64, torch.uint8: sx.SX_U8}
    if tensor.dtype not in m:
        raise TypeError(f"unsupported tensor dtype {tensor.dtype}")
    return m[tensor.dtype]


CUDA_STREAM_LEGACY = 0x1  # the runtime's handle of the legacy default stream (cudaStreamLegacy)


def target_on_torch_stream(device: int = 0, stream=None, budget_bytes: int = 0):
    """A target on ``device`` that enqueues on ``stream`` (default: torch's current stream), so
    that its work is ordered with torch's on that stream.  torch names the legacy default
    stream 0, which the C ABI reads as "create a stream": it is passed as cudaStreamLegacy."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return sx.sx_target_create_ext(device, stream.cuda_stream or CUDA_STREAM_LEGACY, budget_bytes)


def wrap_tensor(target, tensor):
    """Borrow a contiguous CUDA tensor's elements as an ``sx_array`` (not charged, not freed)."""
    if not tensor.is_cuda or not tensor.is_contiguous():
        raise ValueError("wrap_tensor needs a contiguous CUDA tensor")
    return sx.sx_array_wrap(target, dtype_of(tensor), tensor.data_ptr(), tensor.numel())
