"""Thin ctypes binding of libxsum.so: the C ABI of include/xsum.h, same names.

Argument marshalling only: every computation happens in the CUDA library.
Pointer arguments accept plain integers (device or host addresses) or objects
with ``data_ptr()`` (torch tensors); ``stream`` accepts an integer handle, a
``torch.cuda.Stream`` or None (the current torch stream when torch is loaded,
else the legacy default stream). There is no CPU fallback: if the library is
missing or cannot load, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import struct

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libxsum.so")

XS_OK = 0
XS_ERR_INVALID_VALUE = 1
XS_ERR_INVALID_POINTER = 2
XS_ERR_OUT_OF_MEMORY = 3
XS_ERR_CUDA = 4
XS_ERR_TIMEOUT = 5
XS_ERR_BUDGET = 6
XS_ERR_NOT_SUPPORTED = 7
XS_ERR_NOT_READY = 8

XS_METHOD_AUTO = 0
XS_METHOD_SMALL = 1
XS_METHOD_LARGE = 2
XS_ACC_BYTES = 560

_c_int64 = ctypes.c_int64
_vp = ctypes.c_void_p


class XsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class xs_seg_options(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("unroll", ctypes.c_int), ("tile_elems", ctypes.c_int),
                ("short_max", ctypes.c_int), ("carry_tiles", ctypes.c_int)]


class xs_server_options(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_sessions", ctypes.c_int),
                ("streams", ctypes.c_int), ("max_batch", ctypes.c_int), ("tile_elems", ctypes.c_int),
                ("long_min", ctypes.c_int), ("long_tile", ctypes.c_int)]


class xs_request(ctypes.Structure):
    _fields_ = [("session", ctypes.c_uint64), ("d_values", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class xs_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("value", ctypes.c_double),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_launch_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]


class xs_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "batches", "bytes_done",
                                              "queued", "in_flight_bytes", "open_sessions")]


class xs_replay_item(ctypes.Structure):
    _fields_ = [("t_ns", ctypes.c_int64), ("session_tag", ctypes.c_uint64),
                ("d_values", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


XS_REQ_FINISH = 1

# name: (restype, argtypes)
_SIGS = {
    "xs_version": (ctypes.c_char_p, []),
    "xs_get_last_error": (ctypes.c_int, []),
    "xs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "xs_sum": (ctypes.c_double, [_vp, _c_int64, _vp]),
    "xs_sum_ex": (ctypes.c_int, [_vp, _c_int64, _vp, ctypes.POINTER(ctypes.c_double)]),
    "xs_sum_async": (ctypes.c_int, [_vp, _c_int64, _vp, ctypes.c_int, _vp]),
    "xs_sum_async_config": (ctypes.c_int, [_vp, _c_int64, _vp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, _vp]),
    "xs_list_configs": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "xs_set_prefetch_tiles": (ctypes.c_int, [ctypes.c_int]),
    "xs_default_shape": (ctypes.c_int, [_c_int64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "xs_sum_host": (ctypes.c_int, [_vp, _c_int64, ctypes.POINTER(ctypes.c_double), _vp]),
    "xs_sum_noalloc": (ctypes.c_int, [_vp, _c_int64, _vp, _vp]),
    "xs_inexact_sum_async": (ctypes.c_int, [_vp, _c_int64, _vp, _vp]),
    "xs_mean_async": (ctypes.c_int, [_vp, _c_int64, _vp, _vp]),
    "xs_dot_async": (ctypes.c_int, [_vp, _vp, _c_int64, _vp, _vp]),
    "xs_norm2_async": (ctypes.c_int, [_vp, _c_int64, _vp, _vp]),
    "xs_dot_method_async": (ctypes.c_int, [_vp, _vp, _c_int64, _vp, ctypes.c_int, _vp]),
    "xs_norm2_method_async": (ctypes.c_int, [_vp, _c_int64, _vp, ctypes.c_int, _vp]),
    "xs_sum_f32_async": (ctypes.c_int, [_vp, _c_int64, _vp, _vp]),
    "xs_sum_f32_method_async": (ctypes.c_int, [_vp, _c_int64, _vp, ctypes.c_int, _vp]),
    "xs_acc_round_div": (ctypes.c_int, [_vp, _c_int64, _vp, _vp]),
    "xs_autotune_sum": (ctypes.c_int, [_vp, _c_int64, ctypes.c_int, _vp,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "xs_sum_segments": (ctypes.c_int, [_vp, _vp, _c_int64, _vp, _vp]),
    "xs_sum_each_async": (ctypes.c_int, [_vp, _vp, _c_int64, _vp, _vp]),
    "xs_seg_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, _vp, _c_int64, _vp,
                                          ctypes.POINTER(xs_seg_options), _vp]),
    "xs_seg_plan_launch": (ctypes.c_int, [_vp, _vp]),
    "xs_seg_plan_launch_direct": (ctypes.c_int, [_vp, _vp]),
    "xs_seg_plan_kernel_launches": (ctypes.c_int, [_vp]),
    "xs_seg_plan_check": (ctypes.c_int, [_vp, _vp]),
    "xs_seg_plan_destroy": (ctypes.c_int, [_vp]),
    "xs_autotune_segments": (ctypes.c_int, [_vp, _vp, _c_int64, _vp, ctypes.c_int, _vp,
                                            ctypes.POINTER(xs_seg_options),
                                            ctypes.POINTER(ctypes.c_float)]),
    "xs_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(xs_server_options)]),
    "xs_server_open_session": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "xs_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(xs_request), ctypes.POINTER(ctypes.c_uint64)]),
    "xs_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(xs_result)]),
    "xs_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(xs_result)]),
    "xs_server_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(xs_server_stats)]),
    "xs_server_destroy": (ctypes.c_int, [_vp]),
    "xs_server_replay": (ctypes.c_int, [_vp, ctypes.POINTER(xs_replay_item), ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64)]),
    "xs_serial_replay": (ctypes.c_int, [ctypes.POINTER(xs_replay_item), ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                        _vp]),
    "xs_acc_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp]),
    "xs_acc_init": (ctypes.c_int, [_vp, _vp]),
    "xs_acc_add": (ctypes.c_int, [_vp, _vp, _c_int64, _vp]),
    "xs_acc_merge": (ctypes.c_int, [_vp, _vp, _vp]),
    "xs_acc_round": (ctypes.c_int, [_vp, _vp, _vp]),
    "xs_acc_export": (ctypes.c_int, [_vp, _vp, _vp]),
    "xs_acc_import": (ctypes.c_int, [_vp, _vp, _vp]),
    "xs_acc_destroy": (ctypes.c_int, [_vp]),
    "xs_acc_device_state": (_vp, [_vp]),
    "xs_debug_fail_allocation": (ctypes.c_int, [_c_int64]),
    "xs_debug_live_allocations": (_c_int64, []),
    "xs_is_debug_build": (ctypes.c_int, []),
    "xs_debug_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)]),
}

_lib = None


def load(path: str | None = None):
    """Loads libxsum.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libxsum.so not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    return list(_SIGS)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "value"):
        return x.value
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _vals(x, n: int, itemsize: int = 8) -> int | None:
    """Pointer of a values argument. When it is a tensor or an array, n items of
    `itemsize` bytes must lie inside it (ValueError otherwise): a raw address
    can carry no such check, so the library trusts n, and a kernel given an n
    past the end of its buffer would read memory it does not own."""
    if hasattr(x, "numel") and hasattr(x, "element_size"):
        have = x.numel() * x.element_size()
    elif hasattr(x, "nbytes") and hasattr(x, "ctypes"):
        have = x.nbytes
    else:
        return _ptr(x)
    if n * itemsize > have:  # (a negative n is the library's to reject)
        raise ValueError(f"{n} values of {itemsize} bytes do not fit in a buffer of {have} bytes")
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("values must be contiguous")
        return x.data_ptr()
    return x.ctypes.data


_torch = None


def _stream(s) -> int | None:
    global _torch
    if s is None:
        if _torch is None:
            try:
                import torch
            except ImportError:
                return None
            _torch = torch
        # is_initialized() is a flag test; once CUDA is up, torch's current stream
        if _torch.cuda.is_initialized():
            return _torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int, where: str) -> None:
    if status != XS_OK:
        raise XsError(status, where)


def status_string(s: int) -> str:
    return load().xs_status_string(s).decode()


def xs_version() -> str:
    return load().xs_version().decode()


def xs_get_last_error() -> int:
    return load().xs_get_last_error()


def xs_sum(d_values, n: int, stream=None) -> float:
    return load().xs_sum(_vals(d_values, n), n, _stream(stream))


def xs_sum_ex(d_values, n: int, stream=None) -> float:
    out = ctypes.c_double()
    _check(load().xs_sum_ex(_vals(d_values, n), n, _stream(stream), ctypes.byref(out)), "xs_sum_ex")
    return out.value


def xs_sum_async(d_values, n: int, d_out, method: int = XS_METHOD_AUTO, stream=None) -> None:
    _check(load().xs_sum_async(_vals(d_values, n), n, _ptr(d_out), method, _stream(stream)),
           "xs_sum_async")


def xs_sum_async_config(d_values, n: int, d_out, method: int, block: int, unroll: int,
                        grid: int = 0, stream=None) -> None:
    _check(load().xs_sum_async_config(_vals(d_values, n), n, _ptr(d_out), method, block, unroll, grid,
                                      _stream(stream)), "xs_sum_async_config")


def xs_default_shape(n: int) -> dict:
    m, b, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().xs_default_shape(n, ctypes.byref(m), ctypes.byref(b), ctypes.byref(u)),
           "xs_default_shape")
    return {"method": m.value, "block": b.value, "unroll": u.value}


def xs_set_prefetch_tiles(tiles: int) -> None:
    _check(load().xs_set_prefetch_tiles(tiles), "xs_set_prefetch_tiles")


def xs_list_configs() -> list[tuple[int, int, int]]:
    lib = load()
    k = lib.xs_list_configs(None, None, None, 0)
    m = (ctypes.c_int * k)()
    b = (ctypes.c_int * k)()
    u = (ctypes.c_int * k)()
    lib.xs_list_configs(m, b, u, k)
    return [(m[i], b[i], u[i]) for i in range(k)]


def xs_sum_host(h_values, n: int, stream=None) -> float:
    out = ctypes.c_double()
    _check(load().xs_sum_host(_vals(h_values, n), n, ctypes.byref(out), _stream(stream)), "xs_sum_host")
    return out.value


XS_NOALLOC_MAX_TERMS = 1 << 45


def xs_sum_noalloc(d_values, n: int, d_out, stream=None) -> None:
    _check(load().xs_sum_noalloc(_vals(d_values, n), n, _ptr(d_out), _stream(stream)),
           "xs_sum_noalloc")


def xs_mean_async(d_values, n: int, d_out, stream=None) -> None:
    _check(load().xs_mean_async(_vals(d_values, n), n, _ptr(d_out), _stream(stream)), "xs_mean_async")


def xs_dot_async(d_x, d_y, n: int, d_out, stream=None) -> None:
    _check(load().xs_dot_async(_vals(d_x, n), _vals(d_y, n), n, _ptr(d_out), _stream(stream)),
           "xs_dot_async")


def xs_norm2_async(d_x, n: int, d_out, stream=None) -> None:
    _check(load().xs_norm2_async(_vals(d_x, n), n, _ptr(d_out), _stream(stream)), "xs_norm2_async")


def xs_dot_method_async(d_x, d_y, n: int, d_out, method: int, stream=None) -> None:
    _check(load().xs_dot_method_async(_vals(d_x, n), _vals(d_y, n), n, _ptr(d_out), method,
                                      _stream(stream)), "xs_dot_method_async")


def xs_norm2_method_async(d_x, n: int, d_out, method: int, stream=None) -> None:
    _check(load().xs_norm2_method_async(_vals(d_x, n), n, _ptr(d_out), method, _stream(stream)),
           "xs_norm2_method_async")


def xs_sum_f32_async(d_values, n: int, d_out, stream=None) -> None:
    _check(load().xs_sum_f32_async(_vals(d_values, n, 4), n, _ptr(d_out), _stream(stream)),
           "xs_sum_f32_async")


def xs_sum_f32_method_async(d_values, n: int, d_out, method: int, stream=None) -> None:
    _check(load().xs_sum_f32_method_async(_vals(d_values, n, 4), n, _ptr(d_out), method, _stream(stream)),
           "xs_sum_f32_method_async")


def xs_acc_round_div(h: int, divisor: int, d_out, stream=None) -> None:
    _check(load().xs_acc_round_div(h, divisor, _ptr(d_out), _stream(stream)), "xs_acc_round_div")


def xs_inexact_sum_async(d_values, n: int, d_out, stream=None) -> None:
    _check(load().xs_inexact_sum_async(_vals(d_values, n), n, _ptr(d_out), _stream(stream)),
           "xs_inexact_sum_async")


def xs_autotune_sum(d_values, n: int, reps: int = 5, stream=None):
    m, b, u, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(load().xs_autotune_sum(_vals(d_values, n), n, reps, _stream(stream), ctypes.byref(m),
                                  ctypes.byref(b), ctypes.byref(u), ctypes.byref(t)),
           "xs_autotune_sum")
    return {"method": m.value, "block": b.value, "unroll": u.value, "us": t.value}


def xs_sum_segments(d_values, d_offsets, nseg: int, d_out, stream=None) -> None:
    _check(load().xs_sum_segments(_ptr(d_values), _ptr(d_offsets), nseg, _ptr(d_out),
                                  _stream(stream)), "xs_sum_segments")


def xs_sum_each_async(d_values, h_offsets, nseg: int, d_out, stream=None) -> None:
    """h_offsets: a host int64 buffer (numpy array, or an address)."""
    if hasattr(h_offsets, "ctypes"):
        h_offsets = h_offsets.ctypes.data
    _check(load().xs_sum_each_async(_ptr(d_values), _ptr(h_offsets), nseg, _ptr(d_out),
                                    _stream(stream)), "xs_sum_each_async")


def _opts(opts) -> xs_seg_options | None:
    if opts is None:
        return None
    if isinstance(opts, xs_seg_options):
        return opts
    o = xs_seg_options()
    for k, v in dict(opts).items():
        setattr(o, k, int(v))
    return o


def xs_seg_plan_create(d_values, d_offsets, nseg: int, d_out, opts=None, stream=None) -> int:
    h = _vp()
    o = _opts(opts)
    _check(load().xs_seg_plan_create(ctypes.byref(h), _ptr(d_values), _ptr(d_offsets), nseg,
                                     _ptr(d_out), ctypes.byref(o) if o is not None else None,
                                     _stream(stream)), "xs_seg_plan_create")
    return h.value


def xs_seg_plan_launch(plan: int, stream=None) -> None:
    _check(load().xs_seg_plan_launch(plan, _stream(stream)), "xs_seg_plan_launch")


def xs_seg_plan_launch_direct(plan: int, stream=None) -> None:
    _check(load().xs_seg_plan_launch_direct(plan, _stream(stream)), "xs_seg_plan_launch_direct")


def xs_seg_plan_kernel_launches(plan: int) -> int:
    return load().xs_seg_plan_kernel_launches(plan)


def xs_seg_plan_check(plan: int, stream=None) -> None:
    """Raises XsError(XS_ERR_INVALID_VALUE) if the last launch found malformed offsets."""
    _check(load().xs_seg_plan_check(plan, _stream(stream)), "xs_seg_plan_check")


def xs_seg_plan_destroy(plan: int) -> None:
    _check(load().xs_seg_plan_destroy(plan), "xs_seg_plan_destroy")


def xs_autotune_segments(d_values, d_offsets, nseg: int, d_out, reps: int = 3, stream=None):
    o = xs_seg_options()
    t = ctypes.c_float()
    _check(load().xs_autotune_segments(_ptr(d_values), _ptr(d_offsets), nseg, _ptr(d_out), reps,
                                       _stream(stream), ctypes.byref(o), ctypes.byref(t)),
           "xs_autotune_segments")
    return {f: getattr(o, f) for f, _ in xs_seg_options._fields_} | {"us": t.value}


def xs_acc_create(stream=None) -> int:
    h = _vp()
    _check(load().xs_acc_create(ctypes.byref(h), _stream(stream)), "xs_acc_create")
    return h.value


def xs_acc_init(h: int, stream=None) -> None:
    _check(load().xs_acc_init(h, _stream(stream)), "xs_acc_init")


def xs_acc_add(h: int, d_values, n: int, stream=None) -> None:
    _check(load().xs_acc_add(h, _vals(d_values, n), n, _stream(stream)), "xs_acc_add")


def xs_acc_merge(dst: int, src: int, stream=None) -> None:
    _check(load().xs_acc_merge(dst, src, _stream(stream)), "xs_acc_merge")


def xs_acc_round(h: int, d_out, stream=None) -> None:
    _check(load().xs_acc_round(h, _ptr(d_out), _stream(stream)), "xs_acc_round")


def xs_acc_export(h: int, stream=None) -> bytes:
    buf = ctypes.create_string_buffer(XS_ACC_BYTES)
    _check(load().xs_acc_export(h, buf, _stream(stream)), "xs_acc_export")
    return buf.raw


def xs_acc_import(h: int, state: bytes, stream=None) -> None:
    if len(state) != XS_ACC_BYTES:
        raise ValueError("state must be XS_ACC_BYTES long")
    buf = ctypes.create_string_buffer(state, XS_ACC_BYTES)
    _check(load().xs_acc_import(h, buf, _stream(stream)), "xs_acc_import")


def xs_acc_destroy(h: int) -> None:
    _check(load().xs_acc_destroy(h), "xs_acc_destroy")


def xs_acc_device_state(h: int) -> int:
    return load().xs_acc_device_state(h)


def xs_debug_fail_allocation(k: int) -> None:
    _check(load().xs_debug_fail_allocation(k), "xs_debug_fail_allocation")


def xs_debug_live_allocations() -> int:
    return load().xs_debug_live_allocations()


def xs_is_debug_build() -> bool:
    return bool(load().xs_is_debug_build())


def xs_debug_status() -> int:
    """OR of the check codes the debug build's kernels recorded since the last call."""
    v = ctypes.c_uint64()
    _check(load().xs_debug_status(ctypes.byref(v)), "xs_debug_status")
    return v.value


def acc_state_chunks(state: bytes) -> list[int]:
    """The 67 signed chunks of an exported state (little-endian int64)."""
    return list(struct.unpack("<67q", state[:536]))


def _result_dict(r: xs_result) -> dict:
    return {"status": r.status, "value": r.value, "t_submit_ns": r.t_submit_ns,
            "t_admit_ns": r.t_admit_ns, "t_launch_ns": r.t_launch_ns, "t_done_ns": r.t_done_ns}


def xs_server_create(budget_bytes: int = 0, max_sessions: int = 0, streams: int = 0,
                     max_batch: int = 0, tile_elems: int = 0, long_min: int = 0, long_tile: int = 0) -> int:
    o = xs_server_options(budget_bytes, max_sessions, streams, max_batch, tile_elems, long_min, long_tile)
    h = _vp()
    _check(load().xs_server_create(ctypes.byref(h), ctypes.byref(o)), "xs_server_create")
    return h.value


def xs_server_open_session(server: int) -> int:
    sid = ctypes.c_uint64()
    _check(load().xs_server_open_session(server, ctypes.byref(sid)), "xs_server_open_session")
    return sid.value


def xs_server_submit(server: int, d_values, n: int, session: int = 0, flags: int = 0) -> int:
    req = xs_request(session, _vals(d_values, n), n, flags, 0)
    rid = ctypes.c_uint64()
    _check(load().xs_server_submit(server, ctypes.byref(req), ctypes.byref(rid)), "xs_server_submit")
    return rid.value


def xs_server_poll(server: int, request_id: int) -> dict:
    r = xs_result()
    _check(load().xs_server_poll(server, request_id, ctypes.byref(r)), "xs_server_poll")
    return _result_dict(r)


def xs_server_wait(server: int, request_id: int, timeout_ns: int = -1) -> dict:
    r = xs_result()
    _check(load().xs_server_wait(server, request_id, timeout_ns, ctypes.byref(r)), "xs_server_wait")
    return _result_dict(r)


def xs_server_stats_get(server: int) -> dict:
    st = xs_server_stats()
    _check(load().xs_server_stats_get(server, ctypes.byref(st)), "xs_server_stats_get")
    return {f: getattr(st, f) for f, _ in xs_server_stats._fields_}


def xs_server_destroy(server: int) -> None:
    _check(load().xs_server_destroy(server), "xs_server_destroy")


def xs_server_replay(server: int, items) -> tuple[list[int], int]:
    """items: sequence of (t_ns, session_tag, d_values_ptr, n, flags). Returns (ids, start_ns)."""
    arr = _replay_items(items)
    ids = (ctypes.c_uint64 * len(items))()
    start = ctypes.c_int64()
    _check(load().xs_server_replay(server, arr, len(items), ids, ctypes.byref(start)),
           "xs_server_replay")
    return list(ids), start.value


def _replay_items(items):
    arr = (xs_replay_item * len(items))()
    for k, (t, tag, ptr, n, fl) in enumerate(items):
        arr[k] = xs_replay_item(int(t), int(tag), int(ptr), int(n), int(fl), 0)
    return arr


def xs_serial_replay(items, stream=None) -> tuple[list[float], list[int]]:
    """items as for xs_server_replay. Returns (values, done_ns) per item."""
    arr = _replay_items(items)
    vals = (ctypes.c_double * len(items))()
    done = (ctypes.c_int64 * len(items))()
    _check(load().xs_serial_replay(arr, len(items), vals, done, _stream(stream)), "xs_serial_replay")
    return list(vals), list(done)
