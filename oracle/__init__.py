"""Serial CPU oracle of the STREAM hot path (Heller et al., Section 5, Listing 4).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import this package.
It shares no code with the CUDA library (``paper_2206_06302_b300``) and does not import it.

The arithmetic lives in ``stream_oracle.c`` (plain loops, binary64/binary32, compiled with
``-O2 -ffp-contract=off`` and no fast-math); this module only builds it with gcc and passes
numpy arrays to it through ctypes.  Every function here is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (closed forms, hand-derived rounding cases, numpy ufuncs,
invariants); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "stream_oracle.c")
_LIB = os.path.join(_HERE, "libstream_oracle.so")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def compile_library(src: str, out: str, cflags=None) -> str:
    """gcc ``src`` into the shared library ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *(CFLAGS if cflags is None else cflags), src, "-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``stream_oracle.c`` into ``libstream_oracle.so`` if it is missing or stale."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(SOURCE)
    if force or stale:
        compile_library(SOURCE, _LIB)
    return _LIB


def _suffix(*arrs) -> str:
    dt = arrs[0].dtype
    for a in arrs:
        if a.dtype != dt:
            raise TypeError("oracle: mixed dtypes")
        if not a.flags.c_contiguous:
            raise ValueError("oracle: arrays must be C-contiguous")
    if dt == np.float64:
        return "f64"
    if dt == np.float32:
        return "f32"
    raise TypeError(f"oracle: unsupported dtype {dt}")


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class Oracle:
    """The oracle's entry points bound to one compiled copy of ``stream_oracle.c``."""

    def __init__(self, libpath: str):
        lib = ctypes.CDLL(libpath)
        P, N = ctypes.c_void_p, ctypes.c_size_t
        D, I = ctypes.c_double, ctypes.c_int
        for t in ("f64", "f32"):
            getattr(lib, f"oracle_copy_{t}").argtypes = [P, P, N]
            getattr(lib, f"oracle_scale_{t}").argtypes = [P, P, N, D]
            getattr(lib, f"oracle_add_{t}").argtypes = [P, P, P, N]
            getattr(lib, f"oracle_triad_{t}").argtypes = [P, P, P, N, D]
            getattr(lib, f"oracle_stream_{t}").argtypes = [P, P, P, N, D, I]
        lib.oracle_to_upper_u8.argtypes = [P, P, N]
        self.lib = lib
        self.path = libpath

    def copy(self, a, out=None):
        """Listing 4, Copy: ``out = a``."""
        out = np.empty_like(a) if out is None else out
        getattr(self.lib, f"oracle_copy_{_suffix(a, out)}")(_p(a), _p(out), a.size)
        return out

    def scale(self, c, q, out=None):
        """Listing 4, Scale: ``out = c * q``."""
        out = np.empty_like(c) if out is None else out
        getattr(self.lib, f"oracle_scale_{_suffix(c, out)}")(_p(c), _p(out), c.size, q)
        return out

    def add(self, a, b, out=None):
        """Listing 4, Add: ``out = a + b``."""
        out = np.empty_like(a) if out is None else out
        getattr(self.lib, f"oracle_add_{_suffix(a, b, out)}")(_p(a), _p(b), _p(out), a.size)
        return out

    def triad(self, b, c, q, out=None):
        """Listing 4, Triad: ``out = b + c * q`` (product rounded first, then the sum)."""
        out = np.empty_like(b) if out is None else out
        getattr(self.lib, f"oracle_triad_{_suffix(b, c, out)}")(_p(b), _p(c), _p(out), b.size, q)
        return out

    def apply(self, op, x, y, q, out=None):
        """One STREAM kernel by name, library operand convention:
        copy ``out=x``, scale ``out=x*q``, add ``out=x+y``, triad ``out=x+y*q``."""
        if op == "copy":
            return self.copy(x, out)
        if op == "scale":
            return self.scale(x, q, out)
        if op == "add":
            return self.add(x, y, out)
        if op == "triad":
            return self.triad(x, y, q, out)
        raise ValueError(op)

    def stream(self, a, b, c, q=3.0, iters=1):
        """Listing 4's stream(), ``iters`` times, in place on (a, b, c)."""
        getattr(self.lib, f"oracle_stream_{_suffix(a, b, c)}")(
            _p(a), _p(b), _p(c), a.size, q, iters)
        return a, b, c

    def to_upper(self, s):
        """Listing 3's element transform: ASCII upper-casing of a byte array."""
        if s.dtype != np.uint8 or not s.flags.c_contiguous:
            raise TypeError("to_upper: contiguous uint8 array expected")
        out = np.empty_like(s)
        self.lib.oracle_to_upper_u8(_p(s), _p(out), s.size)
        return out


_lock = threading.Lock()
_default: Oracle | None = None


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def copy(a, out=None):
    return default().copy(a, out)


def scale(c, q, out=None):
    return default().scale(c, q, out)


def add(a, b, out=None):
    return default().add(a, b, out)


def triad(b, c, q, out=None):
    return default().triad(b, c, q, out)


def apply(op, x, y, q, out=None):
    return default().apply(op, x, y, q, out)


def stream(a, b, c, q=3.0, iters=1):
    return default().stream(a, b, c, q, iters)


def to_upper(s):
    return default().to_upper(s)
