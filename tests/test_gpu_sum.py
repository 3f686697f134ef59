"""GPU parity of the single-array exact sum against the CPU oracle (bit for bit).

Every compiled launch shape of both methods (per-thread small superaccumulators;
per-block large superaccumulator with transfers) must give the oracle's bits:
the paper's result is the correctly rounded exact sum, which has no tolerance.
"""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import c_oracle
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, f2b, out_slot, to_device
from tests.test_oracle import GOLDEN_CASES

pytestmark = pytest.mark.gpu


def configs():
    xsum.load()
    return xsum.xs_list_configs()


CONFIGS = configs() if True else []
IDS = [f"{'small' if m == 1 else 'large'}-{b}x{u}" for m, b, u in CONFIGS]


def gpu_bits(d, method, block, unroll, grid=0):
    out = out_slot()
    xsum.xs_sum_async_config(d, d.numel(), out, method, block, unroll, grid)
    return int(bits_of(out)[0])


def all_shapes_equal(bits, expect, grids=(0,), misalign=(0,)):
    for mis in misalign:
        d = to_device(bits, mis)
        for m, b, u in CONFIGS:
            for g in grids:
                got = gpu_bits(d, m, b, u, g)
                assert got == expect, (m, b, u, g, mis, hex(got), hex(expect))


def test_cfg0_cancel_all_shapes():
    x = W.f64_to_bits(W.cfg0_cancel(0))
    expect = c_oracle.sum_bits(x)
    all_shapes_equal(x, expect, grids=(0, 1, 2, 7), misalign=(0, 1))


@pytest.mark.parametrize("name,bits,expected", GOLDEN_CASES, ids=[c[0] for c in GOLDEN_CASES])
def test_golden(name, bits, expected):
    all_shapes_equal(np.array(bits, dtype=np.uint64), expected, misalign=(0, 1))


@pytest.mark.parametrize("case", W.cfg2d_side_cases(), ids=[c[0] for c in W.cfg2d_side_cases()])
def test_side_cases(case):
    bits = W.f64_to_bits(np.array(case[1], dtype=np.float64))
    all_shapes_equal(bits, c_oracle.sum_bits(bits), misalign=(0, 1))


SIZES = [1, 2, 3, 5, 31, 32, 33, 255, 1000, 4095, 4096, 4097, 65537, (1 << 20) + 3]


@pytest.mark.parametrize("n", SIZES)
def test_sizes_full_range(n):
    x = W.cfg2a_full_range(n, 0, n)
    all_shapes_equal(x, c_oracle.sum_bits(x), misalign=(0, 1))


@pytest.mark.parametrize("n", [7, 1000, 70001])
def test_sizes_with_specials(n):
    rng = np.random.default_rng(n)
    x = W.cfg1_band(n, 0, n).copy()
    specials = np.array([0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000123,
                         0xFFF4000000000456, 0x8000000000000000, 0], dtype=np.uint64)
    for k in range(4):
        sel = rng.integers(0, n, size=max(1, n // 500))
        x[sel] = specials[rng.integers(0, specials.size, sel.size)]
        all_shapes_equal(x, c_oracle.sum_bits(x))


@pytest.mark.parametrize("gen", ["paired", "cancel", "band", "mirror"])
def test_distributions_mid_size(gen):
    n = 3_000_001
    if gen == "paired":
        x = W.cfg2a_paired(1, 0, n)
    elif gen == "cancel":
        x = W.cfg2b_cancel_1e300(1, 0, n)
    elif gen == "band":
        x = W.cfg1_band(1, 0, n)
    else:
        x = W.f64_to_bits(W.zero_sum_mirror(1, n))
    all_shapes_equal(x, c_oracle.sum_bits(x), grids=(0, 3))


def test_all_negative_zero_and_empty():
    z = np.full(100_000, 0x8000000000000000, dtype=np.uint64)
    all_shapes_equal(z, 0x8000000000000000)
    z[77777] = 0
    all_shapes_equal(z, 0)
    out = out_slot()
    xsum.xs_sum_async(0, 0, out)
    assert int(bits_of(out)[0]) == 0


REPEAT_V = [0.1, 1.0 - 2.0 ** -53, 3 * 5e-324, 1.7976931348623157e308 / 2 ** 30, -0.7]


@pytest.mark.parametrize("N", [2047, 2048, 4095, 4096, 4097, 100003, 1_000_000])
def test_repeat_closed_form(N):
    """N copies of v sum to fl(N*v): carry interval and 4096-add transfer stress."""
    for v in REPEAT_V:
        all_shapes_equal(np.full(N, f2b(v), dtype=np.uint64), f2b(v * N))


@pytest.mark.parametrize("every", [3, 7, 61, 997])
def test_rare_terms_between_largest_chunk_adds(every):
    """Same-sign terms whose significand sits at the top of a chunk (e & 31 ==
    31, the largest high parts, so the chunks approach their bound between
    carry propagations), with zeros and subnormals spread through them: the
    groups holding one go through the short path, are taken back and re-added.
    Exact sums fixed by integer arithmetic: the oracle decides."""
    n = 3_000_017
    rng = np.random.default_rng(every)
    e = np.uint64(0x7DF)  # biased exponent 2015: chunk 62, shift 31
    x = (e << np.uint64(52)) | rng.integers(0, 1 << 52, n, dtype=np.uint64)
    sel = np.arange(every // 2, n, every)
    rare = np.array([0, 0x8000000000000000, 1, 0x800FFFFFFFFFFFFF, 0x0008000000000000],
                    dtype=np.uint64)
    x[sel] = rare[rng.integers(0, rare.size, sel.size)]
    all_shapes_equal(x, c_oracle.sum_bits(x), misalign=(0, 1))
    # the same with one Inf and one NaN among them: only the special record decides
    y = x.copy()
    y[n // 3] = 0x7FF0000000000000
    all_shapes_equal(y, 0x7FF0000000000000)
    y[2 * n // 3] = 0xFFF8000000000321
    all_shapes_equal(y, c_oracle.sum_bits(y))


@pytest.mark.parametrize("frac", [0.01, 0.1, 0.5, 0.97])
def test_many_zeros_of_both_signs(frac):
    """Zeros (+0 and -0) at random positions among band values: a zero in a
    group of the speculative short path is taken back in place (its 2^20 in
    chunk 1); every shape, aligned and not, against the oracle, and the same
    values as floats through both binary32 methods."""
    n = 1_000_003
    rng = np.random.default_rng(int(frac * 1000))
    x = W.cfg1_band(21, 0, n).copy()
    sel = rng.random(n) < frac
    x[sel] = np.where(rng.random(int(sel.sum())) < 0.5, np.uint64(0), np.uint64(0x8000000000000000))
    all_shapes_equal(x, c_oracle.sum_bits(x), misalign=(0, 1))
    f = x.view(np.float64).astype(np.float32)
    f[sel] = np.where(x[sel] >> np.uint64(63), np.float32(-0.0), np.float32(0.0))
    fb = f.view(np.uint32)
    expect = c_oracle.sum_f32_bits(fb)
    d = torch.from_numpy(fb.view(np.int32)).cuda().view(torch.float32)
    o32 = torch.empty(1, dtype=torch.float32, device="cuda")
    for m in (xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE):
        xsum.xs_sum_f32_method_async(d, n, o32, m)
        assert int(o32.view(torch.int32).cpu().numpy().view(np.uint32)[0]) == expect, (frac, m)


def test_permutation_invariance():
    x = W.cfg2a_paired(2, 0, 500_000)
    expect = c_oracle.sum_bits(x)
    rng = np.random.default_rng(0)
    for _ in range(3):
        all_shapes_equal(x[rng.permutation(x.size)], expect)


def test_xs_sum_blocking_forms():
    x = W.cfg0_cancel(3)
    expect = c_oracle.sum_bits(W.f64_to_bits(x))
    d = torch.from_numpy(x).cuda()
    assert f2b(xsum.xs_sum(d, d.numel())) == expect
    assert f2b(xsum.xs_sum_ex(d, d.numel())) == expect
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert f2b(xsum.xs_sum_ex(d, d.numel(), s)) == expect


def test_host_buffer_form():
    for n in [10_000, 30_000_001]:
        x = W.bits_to_f64(W.cfg2a_paired(4, 0, n)) if n > 10_000 else W.cfg0_cancel(1)
        expect = c_oracle.sum_bits(W.f64_to_bits(x))
        h = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        assert f2b(xsum.xs_sum_host(h, h.numel())) == expect
        assert f2b(xsum.xs_sum_host(h, h.numel())) == expect  # workspace reuse


def test_errors():
    out = out_slot()
    d = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_sum_async(d, -1, out)
    assert e.value.status == xsum.XS_ERR_INVALID_VALUE
    h = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_sum_async(h, 10, out)
    assert e.value.status == xsum.XS_ERR_INVALID_POINTER
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_sum_async(d.data_ptr() + 4, 5, out)
    assert e.value.status == xsum.XS_ERR_INVALID_VALUE
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_sum_async_config(d, 10, out, xsum.XS_METHOD_SMALL, 96, 4)
    assert e.value.status == xsum.XS_ERR_NOT_SUPPORTED


def test_inexact_baseline_runs():
    x = W.bits_to_f64(W.cfg1_band(0, 0, 1_000_000))
    d = torch.from_numpy(x).cuda()
    out = out_slot()
    xsum.xs_inexact_sum_async(d, d.numel(), out)
    ref = W.bits_to_f64(np.array([c_oracle.sum_bits(W.f64_to_bits(x))], dtype=np.uint64))[0]
    assert abs(float(out.item()) - ref) <= 1e-6 * np.abs(x).sum()


def test_autotune_then_auto_is_exact():
    x = W.cfg1_band(5, 0, 5_000_000)
    d = to_device(x)
    r = xsum.xs_autotune_sum(d, d.numel(), reps=3)
    assert r["method"] in (1, 2) and r["us"] > 0
    out = out_slot()
    xsum.xs_sum_async(d, d.numel(), out)
    assert int(bits_of(out)[0]) == c_oracle.sum_bits(x)


# ----------------------------- full-size configurations ---------------------

def _default_and_methods(x_dev, expect):
    out = out_slot()
    for method in (xsum.XS_METHOD_AUTO, xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE):
        xsum.xs_sum_async(x_dev, x_dev.numel(), out, method)
        assert int(bits_of(out)[0]) == expect, method


def test_full_cfg1_band_1e8():
    x = W.cfg1_band(0, 0, 10 ** 8)
    expect = c_oracle.sum_bits(x)
    d = to_device(x)
    _default_and_methods(d, expect)


@pytest.mark.parametrize("which", ["full_range", "paired", "cancel_1e300"])
def test_full_cfg2_2e28(which):
    n = 1 << 28
    if which == "full_range":
        x = W.cfg2a_full_range(0, 0, n)
    elif which == "paired":
        x = W.cfg2a_paired(0, 0, n)
    else:
        x = W.cfg2b_cancel_1e300(0, 0, n)
    expect = c_oracle.sum_bits(x)
    d = to_device(x)
    del x
    _default_and_methods(d, expect)


@pytest.mark.parametrize("v", [0.1, 1.0 - 2.0 ** -53, 3 * 5e-324, 1.7976931348623157e308 / 2 ** 30])
def test_full_cfg2c_1e8_copies(v):
    N = 10 ** 8
    d = torch.full((N,), v, dtype=torch.float64, device="cuda")
    _default_and_methods(d, f2b(v * N))
