"""The C ABI library loads and exports every symbol include/xsum.h declares (no GPU calls)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xsum.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(xs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_t")))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1505_05571_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["xs_sum", "xs_sum_ex", "xs_sum_async", "xs_sum_segments", "xs_acc_create",
                 "xs_acc_add", "xs_acc_merge", "xs_acc_round", "xs_acc_export", "xs_acc_import",
                 "xs_acc_destroy", "xs_get_last_error", "xs_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(xs_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1505_05571_gb300 import xsum
    lib = xsum.load()
    for n in declared_functions():
        assert hasattr(lib, n)
        assert n in xsum.declared_symbols(), n


def test_status_strings(lib_path):
    from paper_1505_05571_gb300 import xsum
    assert xsum.status_string(0) == "ok"
    assert "invalid" in xsum.status_string(1)
    assert xsum.xs_version().startswith("xsum-gb300")


def test_compute_fails_loudly_without_gpu(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1505_05571_gb300 import xsum
    with pytest.raises(xsum.XsError):
        xsum.xs_sum_ex(0x1000, 10, None)
    assert xsum.xs_get_last_error() != 0


def test_listed_configs(lib_path):
    from paper_1505_05571_gb300 import xsum
    cfgs = xsum.xs_list_configs()
    assert {m for m, _, _ in cfgs} == {xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE}


def test_no_oracle_in_product():
    """The library package never imports the oracle (no CPU fallback path)."""
    pkg = os.path.join(ROOT, "paper_1505_05571_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".hpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower().replace("no oracle", ""), f


def test_prefetch_setting_range(lib_path):
    """The prefetch knob takes -1 (built-in distances) .. 64 and rejects the rest
    (host-side state only, no GPU call)."""
    from paper_1505_05571_gb300 import xsum
    for bad in (-2, 65, 1 << 20):
        with pytest.raises(xsum.XsError):
            xsum.xs_set_prefetch_tiles(bad)
    for ok in (0, 5, 64, -1):
        xsum.xs_set_prefetch_tiles(ok)


def test_argument_errors_come_before_any_device_work(lib_path):
    """The documented error contract of the boundary, for arguments the host can
    judge alone: it holds with or without a GPU, since no device call is made."""
    import math

    from paper_1505_05571_gb300 import xsum

    def status_of(fn):
        try:
            fn()
        except xsum.XsError as e:
            return e.status
        return xsum.XS_OK

    E_VAL, E_PTR = xsum.XS_ERR_INVALID_VALUE, xsum.XS_ERR_INVALID_POINTER
    cases = [
        (lambda: xsum.xs_sum_ex(0x1000, -1), E_VAL),            # n < 0
        (lambda: xsum.xs_sum_ex(0x1001, 10), E_VAL),            # not 8-byte aligned
        (lambda: xsum.xs_sum_ex(0, 10), E_PTR),                 # null values
        (lambda: xsum.xs_sum_host(0x1000, -3), E_VAL),
        (lambda: xsum.xs_sum_host(0, 5), E_PTR),
        (lambda: xsum.xs_sum_host(0x1004, 5), E_VAL),
        (lambda: xsum.xs_sum_segments(0x1000, 0x2000, -1, 0x3000), E_VAL),
        (lambda: xsum.xs_acc_add(0, 0x1000, 10), E_PTR),        # null handle
        (lambda: xsum.xs_sum_f32_async(0x1000, -1, 0x2000), E_VAL),
        (lambda: xsum.xs_sum_f32_async(0x1000, (1 << 39) + 1, 0x2000), E_VAL),
        (lambda: xsum.xs_sum_f32_method_async(0x1000, 10, 0x2000, 3), E_VAL),  # unknown method
        (lambda: xsum.xs_dot_method_async(0x1000, 0x2000, 10, 0x3000, 3), E_VAL),
        (lambda: xsum.xs_dot_method_async(0x1000, 0x2000, 10, 0x3000, -1), E_VAL),
        (lambda: xsum.xs_norm2_method_async(0x1000, 10, 0x3000, 7), E_VAL),
        (lambda: xsum.xs_dot_async(0x1000, 0x2000, -1, 0x3000), E_VAL),
    ]
    for k, (fn, want) in enumerate(cases):
        assert status_of(fn) == want, k
    # empty inputs need no device either: +0 (the empty sum) and a no-op
    assert xsum.xs_sum_ex(0x1000, 0) == 0.0 and math.copysign(1.0, xsum.xs_sum_ex(0, 0)) == 1.0
    assert xsum.xs_sum_host(0, 0) == 0.0
    xsum.xs_sum_segments(0x1000, 0x2000, 0, 0x3000)
    # the blocking form reports through a quiet NaN and the thread's last error
    assert math.isnan(xsum.xs_sum(0x1000, -1)) and xsum.xs_get_last_error() == E_VAL


def test_binding_rejects_counts_past_the_buffer(lib_path):
    """Given a tensor or an array, the binding refuses an n whose values would
    run past its end (raw addresses carry no extent, so the library cannot
    check this itself); an n that fits goes through to the library."""
    import numpy as np
    import torch

    from paper_1505_05571_gb300 import xsum

    t = torch.zeros(10, dtype=torch.float64)
    a = np.zeros(6, dtype=np.float64)
    f = torch.zeros(9, dtype=torch.float32)
    for call in (lambda: xsum.xs_sum_ex(t, 11), lambda: xsum.xs_sum_host(a, 7),
                 lambda: xsum.xs_sum_async(t[2:], 9, 0x1000), lambda: xsum.xs_dot_async(t, t[1:], 10, 0x1000),
                 lambda: xsum.xs_sum_f32_async(f, 10, 0x1000), lambda: xsum.xs_acc_add(0, t, 11),
                 lambda: xsum.xs_sum_ex(torch.zeros(4, 4, dtype=torch.float64).t(), 16)):
        with pytest.raises(ValueError):
            call()
    assert xsum.xs_sum_ex(t, 0) == 0.0  # fits: the library's empty sum
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_sum_ex(t, -1)  # negative: the library's own error
    assert e.value.status == xsum.XS_ERR_INVALID_VALUE


def test_release_build_has_no_debug_checks(lib_path):
    """The release library reports itself as such, and its debug status is 0
    without any device call."""
    from paper_1505_05571_gb300 import xsum

    assert not xsum.xs_is_debug_build()
    assert xsum.xs_debug_status() == 0
