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
