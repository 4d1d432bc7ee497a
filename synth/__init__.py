"""Seeded synthetic inputs for the embedded-gasket workloads.

This module is the one piece shared by the CPU oracle and the CUDA path: it
produces input values and nothing else.  It holds none of the method's
arithmetic (no membership test, no map, no update rule); every cell of the
n x n embedding gets a value, and each side decides for itself which cells
belong to the gasket.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser published
by S. Vigna as splitmix64.c).  A stream seeded with ``s`` emits, as its
``i``-th output (i = 0, 1, ...), ``mix(s + (i + 1) * GAMMA mod 2**64)``.
The value of cell (x, y) of an n x n embedding is output number ``y * n + x``
of the stream seeded with ``seed``, so any window of the array can be produced
on its own and agrees with the whole-array fill.

Distributions (all exact in both FP32 and FP64):

* ``bernoulli``: ``h >> 63`` as uint8 (0 or 1, p = 1/2);
* ``uniform``:   ``(h >> 40) * 2**-24`` in [0, 1), 24 significant bits;
* ``uniform_affine(lo, width)``: ``lo + width * uniform``; callers keep
  ``lo`` and ``width`` to values that make this exact (e.g. 0.5 and 1.0).

The device-side twin lives in ``synth/synth.cu`` (built to
``synth/libsynth.so``); a GPU test checks the two bit for bit.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream offsets used by the workloads: the state, the conductivity field and
# the loss target draw from seed, seed + 1 and seed + 2.
STREAM_STATE = 0
STREAM_KAPPA = 1
STREAM_TARGET = 2


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """Output number ``index`` (uint64 array) of the stream seeded with ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GAMMA
    return _mix(state)


def cell_hash(seed: int, n: int, x0: int, y0: int, w: int, h: int) -> np.ndarray:
    """Raw 64-bit hash of every cell of the window [x0, x0+w) x [y0, y0+h).

    Returns an (h, w) uint64 array; row index is y - y0, column x - x0.
    """
    ys = np.arange(y0, y0 + h, dtype=np.uint64)[:, None]
    xs = np.arange(x0, x0 + w, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        counter = ys * np.uint64(n) + xs
    return splitmix64(seed, counter)


def bernoulli_u8(seed: int, n: int, x0: int = 0, y0: int = 0,
                 w: Optional[int] = None, h: Optional[int] = None) -> np.ndarray:
    """uint8 0/1 values of the window (defaults to the whole n x n array)."""
    w = n - x0 if w is None else w
    h = n - y0 if h is None else h
    return (cell_hash(seed, n, x0, y0, w, h) >> np.uint64(63)).astype(np.uint8)


def uniform_f32(seed: int, n: int, x0: int = 0, y0: int = 0,
                w: Optional[int] = None, h: Optional[int] = None,
                lo: float = 0.0, width: float = 1.0) -> np.ndarray:
    """float32 values lo + width * U[0,1) of the window (exact for lo=0/0.5, width=1)."""
    w = n - x0 if w is None else w
    h = n - y0 if h is None else h
    u = (cell_hash(seed, n, x0, y0, w, h) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    return (lo + width * u).astype(np.float32)


def values_at(seed: int, n: int, xs: np.ndarray, ys: np.ndarray, dist: str = "uniform",
              lo: float = 0.0, width: float = 1.0) -> np.ndarray:
    """Values of the cells (xs[i], ys[i]) only (same numbers as the window functions)."""
    xs = np.asarray(xs, dtype=np.uint64)
    ys = np.asarray(ys, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = splitmix64(seed, ys * np.uint64(n) + xs)
    if dist == "bernoulli":
        return (h >> np.uint64(63)).astype(np.uint8)
    u = (h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    return (lo + width * u).astype(np.float32)


# --------------------------------------------------------------------------
# Device twin (CUDA).  Loaded lazily; only GPU tests and the benchmark use it.
# --------------------------------------------------------------------------
SYNTH_BERNOULLI_U8 = 0
SYNTH_UNIFORM_F32 = 1

_lib = None


def _lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth.so")


def load_device_lib():
    """Load ``libsynth.so``; raises if it was not built."""
    global _lib
    if _lib is None:
        path = _lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
        lib = ctypes.CDLL(path)
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_fill.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                   ctypes.c_uint64, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_void_p]
        _lib = lib
    return _lib


def device_fill(dev_ptr: int, dist: int, n: int, seed: int, lo: float = 0.0,
                width: float = 1.0, stream: int = 0) -> None:
    """Fill an n x n device array with the same values the host functions give."""
    rc = load_device_lib().synth_fill(ctypes.c_void_p(dev_ptr), dist, n, seed & 0xFFFFFFFFFFFFFFFF,
                                      lo, width, ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError(f"synth_fill failed with status {rc}")
