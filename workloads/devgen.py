"""Device twin of the generators (libxsgen.so), for inputs generated in HBM.

Same formulas as workloads/gen.py; a GPU test compares the two bit for bit.
"""

from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

from . import gen

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "xsgen.cu")
_OUT = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT, "libxsgen.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([exe, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i64, vp, ci = ctypes.c_uint64, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_int
        lib.xsg_band.argtypes = [vp, i64, i64, u64, u64, ci, ci, vp]
        lib.xsg_full_range.argtypes = [vp, i64, i64, u64, u64, vp]
        lib.xsg_paired.argtypes = [vp, i64, i64, u64, u64, u64, u64, ci, u64, u64, vp]
        lib.xsg_cancel.argtypes = [vp, i64, i64, u64, u64, u64, u64, ci, u64, u64, vp]
        for f in (lib.xsg_band, lib.xsg_full_range, lib.xsg_paired, lib.xsg_cancel):
            f.restype = ci
        _lib = lib
    return _lib


def _ok(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"{what}: CUDA error {rc}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def band(out, seed: int, start: int, lo: int = -60, hi: int = 60, stream=None) -> None:
    """out (int64/float64 CUDA tensor) <- cfg1_band(seed, start, out.numel(), lo, hi)."""
    _ok(_load().xsg_band(out.data_ptr(), start, out.numel(), gen.stream_key(seed, "sm"),
                         gen.stream_key(seed, "exp"), lo, hi, _stream(stream)), "xsg_band")


def full_range(out, seed: int, start: int, stream=None) -> None:
    _ok(_load().xsg_full_range(out.data_ptr(), start, out.numel(), gen.stream_key(seed, "sm"),
                               gen.stream_key(seed, "exp"), _stream(stream)), "xsg_full_range")


def paired(out, seed: int, start: int, n_log2: int = 28, stream=None) -> None:
    a_inv, b = gen.affine_constants(seed, n_log2)
    _ok(_load().xsg_paired(out.data_ptr(), start, out.numel(), gen.stream_key(seed, "sm"),
                           gen.stream_key(seed, "exp"), gen.stream_key(seed, "sm2"),
                           gen.stream_key(seed, "exp2"), n_log2, a_inv, b, _stream(stream)),
        "xsg_paired")


def cancel(out, seed: int, start: int, n_log2: int = 28, stream=None) -> None:
    a_inv, b = gen.affine_constants(seed, n_log2)
    _ok(_load().xsg_cancel(out.data_ptr(), start, out.numel(), gen.stream_key(seed, "sm"),
                           gen.stream_key(seed, "exp"), gen.stream_key(seed, "sm2"),
                           gen.stream_key(seed, "exp2"), n_log2, a_inv, b, _stream(stream)),
        "xsg_cancel")
