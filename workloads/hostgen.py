"""Multithreaded host twin of the band generator (libxsgen_host.so).

Same formula as ``workloads.gen.cfg1_band``; a CPU test compares the two bit
for bit. Used where a test regenerates tens of GB of inputs on the host.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import gen

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "xsgen_host.c")
_OUT = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT, "libxsgen_host.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.xgh_band.restype = None
        lib.xgh_band.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
        _lib = lib
    return _lib


def band(seed: int, start: int, count: int, lo: int = -60, hi: int = 60,
         out: np.ndarray | None = None) -> np.ndarray:
    """``cfg1_band(seed, start, count, lo, hi)`` (uint64 bits), on every host core."""
    if out is None:
        out = np.empty(count, dtype=np.uint64)
    assert out.dtype == np.uint64 and out.flags.c_contiguous and out.size >= count
    if count:
        _load().xgh_band(out.ctypes.data, start, count, gen.stream_key(seed, "sm"),
                         gen.stream_key(seed, "exp"), lo, hi)
    return out[:count]
