"""ctypes loader for the plain-C oracle ``xsum_oracle.c`` (test infrastructure only).

``build()`` compiles it with gcc into ``oracle/_build/``; ``load()`` builds on
first use when the shared object is missing or older than the source.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xsum_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libxsum_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.xo_sum_bits.restype = ctypes.c_uint64
        lib.xo_sum_bits.argtypes = [u64p, ctypes.c_int64]
        lib.xo_sum_segments_bits.restype = None
        lib.xo_sum_segments_bits.argtypes = [u64p, i64p, i64p, ctypes.c_int64, u64p]
        lib.xo_max_threads.restype = ctypes.c_int
        lib.xo_sum_f32_bits.restype = ctypes.c_uint32
        lib.xo_sum_f32_bits.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64]
        lib.xo_mean_bits.restype = ctypes.c_uint64
        lib.xo_mean_bits.argtypes = [u64p, ctypes.c_int64]
        _lib = lib
    return _lib


def _u64ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _i64ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def sum_bits(bits: np.ndarray) -> int:
    """Bits of the correctly rounded exact sum of a uint64 (or float64) array."""
    a = np.ascontiguousarray(bits).view(np.uint64)
    return int(load().xo_sum_bits(_u64ptr(a), a.size))


def segment_sums_bits(bits: np.ndarray, offsets: np.ndarray, seg_ids=None) -> np.ndarray:
    """Exact sums (bits) of CSR segments; ``seg_ids`` selects a subset."""
    a = np.ascontiguousarray(bits).view(np.uint64)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    if seg_ids is None:
        seg_ids = np.arange(off.size - 1, dtype=np.int64)
    ids = np.ascontiguousarray(seg_ids, dtype=np.int64)
    out = np.zeros(ids.size, dtype=np.uint64)
    load().xo_sum_segments_bits(_u64ptr(a), _i64ptr(off), _i64ptr(ids), ids.size, _u64ptr(out))
    return out


def max_threads() -> int:
    return int(load().xo_max_threads())


def mean_bits(bits: np.ndarray) -> int:
    """Bits of the correctly rounded exact mean of a uint64 (or float64) array."""
    a = np.ascontiguousarray(bits).view(np.uint64)
    return int(load().xo_mean_bits(_u64ptr(a), a.size))


def sum_f32_bits(bits32: np.ndarray) -> int:
    """Bits of the correctly rounded exact float sum of a uint32 (or float32) array."""
    a = np.ascontiguousarray(bits32).view(np.uint32)
    return int(load().xo_sum_f32_bits(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), a.size))
