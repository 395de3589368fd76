"""Seeded synthetic inputs for the STREAM arrays and for the batched and served workloads.

This module is shared by the oracle-side tests and the CUDA-side tests and by ``bench.py``.
It holds none of the STREAM arithmetic (no copy, scale, add or triad); it only draws numbers.

Generator
---------
SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), in the 64-bit form with the variant-13 finaliser that S. Vigna publishes as
``splitmix64.c``: the state advances by the odd constant GAMMA and each output is the finaliser
``mix64`` of the new state.  Used counter-style: ``word(seed, i)`` is the (i+1)-th output of a
SplitMix64 started from state ``seed``, i.e. ``mix64(seed + (i + 1) * GAMMA mod 2**64)``, so any
element can be drawn independently of the others.  The CUDA library implements the same
definition on the device (its seeded bulk construction); tests check the two agree bit for bit.

Real values
-----------
* FP64: ``u = (w >> 11) * 2**-53`` (exact, in [0, 1)), ``x = RN(lo + RN(RN(hi - lo) * u))``.
* FP32: ``u = (w >> 40) * 2**-24`` (exact), same formula evaluated in binary32 with
  ``lo``/``hi`` first rounded to binary32.
For lo=-1, hi=1 both steps are exact, so x is a multiple of 2**-52 (2**-23) in [-1, 1).

Array seeds
-----------
Array ``k`` (a=0, b=1, c=2) of instance ``j`` under base seed ``S`` uses
``array_seed(S, k, j) = word(word(S, j), k)``.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

#: Default base seed of every synthetic workload in this repository.
BASE_SEED = 20260603


def mix64_scalar(z: int) -> int:
    """SplitMix64 finaliser on one Python int (mod 2**64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def word_scalar(seed: int, i: int) -> int:
    """The (i+1)-th SplitMix64 output from state ``seed``."""
    return mix64_scalar((seed + (i + 1) * GAMMA) & MASK64)


def words_at(seed: int, idx) -> np.ndarray:
    """SplitMix64 words for the element indices ``idx`` (any integer array)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def words(seed: int, n: int, start: int = 0) -> np.ndarray:
    return words_at(seed, np.arange(start, start + n, dtype=np.uint64))


def array_seed(base_seed: int, array_id: int, instance: int = 0) -> int:
    """Seed of array ``array_id`` (a=0, b=1, c=2) of instance ``instance``."""
    return word_scalar(word_scalar(base_seed, instance), array_id)


def _to_f64(w: np.ndarray, lo: float, hi: float) -> np.ndarray:
    u = (w >> np.uint64(11)).astype(np.float64) * np.float64(2.0 ** -53)
    span = np.float64(hi) - np.float64(lo)
    return np.add(np.float64(lo), np.multiply(span, u))


def _to_f32(w: np.ndarray, lo: float, hi: float) -> np.ndarray:
    u = (w >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)
    lo32, hi32 = np.float32(lo), np.float32(hi)
    span = np.float32(hi32 - lo32)
    return np.add(lo32, np.multiply(span, u, dtype=np.float32), dtype=np.float32)


def uniform(seed: int, n: int, dtype, lo: float = -1.0, hi: float = 1.0,
            start: int = 0) -> np.ndarray:
    """Elements [start, start+n) of the seeded uniform array in ``dtype`` (float32/float64)."""
    return uniform_at(seed, np.arange(start, start + n, dtype=np.uint64), dtype, lo, hi)


def uniform_at(seed: int, idx, dtype, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """The seeded uniform values at element indices ``idx``."""
    w = words_at(seed, idx)
    dt = np.dtype(dtype)
    if dt == np.float64:
        return _to_f64(w, lo, hi)
    if dt == np.float32:
        return _to_f32(w, lo, hi)
    raise ValueError(f"unsupported dtype {dt}")


def stream_arrays(n: int, dtype, base_seed: int = BASE_SEED, instance: int = 0):
    """Seeded (a, b, c) arrays, uniform in [-1, 1), for one STREAM instance."""
    return tuple(uniform(array_seed(base_seed, k, instance), n, dtype) for k in range(3))


def closed_form_arrays(n: int, dtype):
    """STREAM's classic start values a=1, b=2, c=0."""
    dt = np.dtype(dtype)
    return (np.full(n, 1.0, dt), np.full(n, 2.0, dt), np.zeros(n, dt))


# --------------------------------------------------------------------------------------
# Workload shapes (batched instances, served requests)
# --------------------------------------------------------------------------------------

def log_uniform_lengths(seed: int, count: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    """``round(2**U)`` with U uniform in [lo_exp, hi_exp), one per item."""
    u = (words(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    e = lo_exp + (hi_exp - lo_exp) * u
    return np.rint(np.exp2(e)).astype(np.int64)


def batched_instances(seed: int = BASE_SEED, count: int = 4096, lo_exp: float = 10,
                      hi_exp: float = 22, ops=("triad", "add")):
    """Independent instances for the batched launcher: (op, n) per instance.

    Ops are drawn uniformly from ``ops``; lengths are log-uniform in [2**lo_exp, 2**hi_exp].
    """
    s_ops = word_scalar(seed, 101)
    s_len = word_scalar(seed, 102)
    op_idx = (words(s_ops, count) % np.uint64(len(ops))).astype(np.int64)
    n = log_uniform_lengths(s_len, count, lo_exp, hi_exp)
    return [(ops[int(k)], int(m)) for k, m in zip(op_idx, n)]


def poisson_requests(seed: int, count: int, rate_per_s: float, lo_exp: float = 12,
                     hi_exp: float = 28, ops=("copy", "scale", "add", "triad"),
                     dtypes=("f64", "f32")):
    """A seeded Poisson request stream.

    Returns a list of dicts with ``t`` (arrival time in seconds from 0; exponential gaps of
    mean 1/rate), ``op``, ``dtype`` and ``n`` (log-uniform in [2**lo_exp, 2**hi_exp]) and
    ``seed`` (the request's own input seed).
    """
    s_gap, s_op, s_dt, s_len, s_in = (word_scalar(seed, 201 + k) for k in range(5))
    u = (words(s_gap, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    gaps = -np.log1p(-u) / rate_per_s
    t = np.cumsum(gaps) - gaps[0]
    op_idx = (words(s_op, count) % np.uint64(len(ops))).astype(np.int64)
    dt_idx = (words(s_dt, count) % np.uint64(len(dtypes))).astype(np.int64)
    n = log_uniform_lengths(s_len, count, lo_exp, hi_exp)
    seeds = words(s_in, count)
    return [dict(t=float(t[k]), op=ops[int(op_idx[k])], dtype=dtypes[int(dt_idx[k])],
                 n=int(n[k]), seed=int(seeds[k])) for k in range(count)]


def mean_log_uniform(lo_exp: float, hi_exp: float) -> float:
    """Mean of 2**U for U uniform in [lo_exp, hi_exp)."""
    return (2.0 ** hi_exp - 2.0 ** lo_exp) / ((hi_exp - lo_exp) * math.log(2.0))
