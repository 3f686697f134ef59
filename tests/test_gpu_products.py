"""GPU parity of the exact dot product and squared norm (fused multiply + exact sum)."""

import numpy as np
import pytest

import workloads as W
from oracle import products
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, out_slot, to_device

pytestmark = pytest.mark.gpu


METHODS = (xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE)


def gpu_dot(x, y, mx=0, my=0):
    """The dot product through the default entry point and through each
    method; all of them must give the same bits, which are returned."""
    dx, dy = to_device(x, mx), to_device(y, my)
    out = out_slot()
    xsum.xs_dot_async(dx, dy, dx.numel(), out)
    got = int(bits_of(out)[0])
    for m in METHODS:
        xsum.xs_dot_method_async(dx, dy, dx.numel(), out, m)
        assert int(bits_of(out)[0]) == got, ("method", m, mx, my)
    return got


def gpu_norm2(x, mx=0):
    dx = to_device(x, mx)
    out = out_slot()
    xsum.xs_norm2_async(dx, dx.numel(), out)
    got = int(bits_of(out)[0])
    for m in METHODS:
        xsum.xs_norm2_method_async(dx, dx.numel(), out, m)
        assert int(bits_of(out)[0]) == got, ("method", m, mx)
    return got


def test_products_reject_unknown_methods():
    dx = to_device(W.cfg1_band(2, 0, 100))
    out = out_slot()
    for bad in (-1, 3):
        with pytest.raises(xsum.XsError):
            xsum.xs_dot_method_async(dx, dx, 100, out, bad)
        with pytest.raises(xsum.XsError):
            xsum.xs_norm2_method_async(dx, 100, out, bad)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 1537, 100_001, 3_000_003])
def test_dot_and_norm_sizes_and_alignments(n):
    x = W.cfg1_band(n, 0, n, -300, 300)
    y = W.cfg2a_full_range(n + 1, 0, n)
    y[((y >> np.uint64(52)) & np.uint64(0x7FF)) > np.uint64(1500)] = 0  # keep most products finite
    expect_dot = products.dot_bits(x, y)
    for mx, my in ((0, 0), (1, 0), (0, 1), (1, 1)):
        assert gpu_dot(x, y, mx, my) == expect_dot, (mx, my)
    expect_n2 = products.norm2_bits(x)
    assert gpu_norm2(x) == expect_n2 and gpu_norm2(x, 1) == expect_n2


def test_products_with_specials_and_subnormals():
    rng = np.random.default_rng(3)
    n = 50_001
    x = W.cfg2a_full_range(31, 0, n).copy()
    y = W.cfg2a_full_range(32, 0, n).copy()
    sel = rng.integers(0, n, 20)
    x[sel[:10]] = np.array([0x7FF0000000000000, 0x7FF8000000000042, 0, 0x8000000000000000,
                            0xFFF0000000000000] * 2, dtype=np.uint64)
    assert gpu_dot(x, y) == products.dot_bits(x, y)
    assert gpu_norm2(x) == products.norm2_bits(x)
    tiny = W.cfg1_band(33, 0, n, -1074 + 52, -520)  # products underflow to subnormals and zero
    assert gpu_dot(tiny, tiny[::-1].copy()) == products.dot_bits(tiny, tiny[::-1].copy())


def test_dot_with_ones_equals_sum():
    x = W.cfg2a_paired(4, 0, 1_000_000)
    ones = np.full(x.size, np.array([1.0]).view(np.uint64)[0], dtype=np.uint64)
    out = out_slot()
    dx = to_device(x)
    xsum.xs_sum_async(dx, dx.numel(), out)
    assert gpu_dot(x, ones) == int(bits_of(out)[0])


def test_full_size_norm_and_dot():
    n = 10 ** 8
    x = W.cfg1_band(0, 0, n)
    y = W.cfg1_band(1, 0, n)
    assert gpu_norm2(x) == products.norm2_bits(x)
    assert gpu_dot(x, y) == products.dot_bits(x, y)


def test_products_underflowing_and_overflowing_in_runs():
    """Products that underflow to zero or a subnormal, or overflow to Inf, in
    every group position: each is taken back from the short path and re-added
    by the general one; the sum must stay the oracle's."""
    n = 1_000_003
    rng = np.random.default_rng(11)
    x = W.cfg1_band(11, 0, n).copy()
    y = W.cfg1_band(12, 0, n).copy()
    tiny = np.array([0x0010000000000000, 0x8000000000000001, 0x3CB0000000000000], dtype=np.uint64)
    sel = np.arange(5, n, 13)
    x[sel] = tiny[rng.integers(0, tiny.size, sel.size)]
    # 2^-53, 2^-2, 0.75: products underflow to zero or land on subnormals
    ys = np.array([0x3CA0000000000000, 0x3FD0000000000000, 0x3FE8000000000000], dtype=np.uint64)
    y[sel] = ys[rng.integers(0, ys.size, sel.size)]
    assert gpu_dot(x, y) == products.dot_bits(x, y)
    assert gpu_dot(x, y, 1, 0) == products.dot_bits(x, y)
    big = x.copy()
    big[7] = np.uint64(0x7FE0000000000000)
    yb = y.copy()
    yb[7] = np.uint64(0x7FE0000000000000)  # overflows to +Inf
    assert gpu_dot(big, yb) == products.dot_bits(big, yb) == 0x7FF0000000000000
