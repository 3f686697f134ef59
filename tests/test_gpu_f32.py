"""GPU parity of the binary32 exact sum against the oracle (bit for bit), for
the default choice and each method: per-thread small superaccumulators and the
per-block large superaccumulator (one chunk per sign+exponent, a column of
words per lane)."""

import numpy as np
import pytest
import torch

from oracle import c_oracle
from tests.test_oracle32 import GOLDEN32, rand32
from paper_1505_05571_gb300 import xsum

pytestmark = pytest.mark.gpu


METHODS = (xsum.XS_METHOD_AUTO, xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE)


def gpu32(bits, misalign=0, method=None):
    """The sum by every method (all must agree); or by one method."""
    a = np.ascontiguousarray(bits, dtype=np.uint32).view(np.int32)
    t = torch.empty(a.size + misalign, dtype=torch.int32, device="cuda")
    if a.size:
        t[misalign:].copy_(torch.from_numpy(a))
    d = t[misalign:].view(torch.float32)
    got = set()
    for m in (METHODS if method is None else (method,)):
        out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        if m == xsum.XS_METHOD_AUTO:
            xsum.xs_sum_f32_async(d, d.numel(), out)
        else:
            xsum.xs_sum_f32_method_async(d, d.numel(), out, m)
        got.add(int(out.view(torch.int32).cpu().numpy().view(np.uint32)[0]))
    assert len(got) == 1, [hex(g) for g in got]
    return got.pop()


@pytest.mark.parametrize("bits,expected,why", GOLDEN32)
def test_golden(bits, expected, why):
    for mis in range(4):
        assert gpu32(np.array(bits, dtype=np.uint32), mis) == expected


@pytest.mark.parametrize("n", [1, 3, 4, 5, 7, 2049, 65536 + 3, 3_000_001])
def test_sizes_and_alignments(n):
    for x in (rand32(n, n), rand32(n + 1, n, -30, 30), rand32(n + 2, n, -149, -120, specials=True)):
        expect = c_oracle.sum_f32_bits(x)
        for mis in (0, 1, 2, 3):
            assert gpu32(x, mis) == expect, mis


@pytest.mark.parametrize("N", [255, 256, 257, 4096, 1_000_001])
def test_repeats(N):
    for v in (0.1, -3.0e38, 1.4e-45):
        b = np.full(N, np.array([v], dtype=np.float32).view(np.uint32)[0], dtype=np.uint32)
        assert gpu32(b) == c_oracle.sum_f32_bits(b)


def test_full_size_2e8():
    x = rand32(0, 2 * 10 ** 8, -60, 60)
    assert gpu32(x) == c_oracle.sum_f32_bits(x)


def test_one_exponent_per_lane_column_carries():
    """2^25 copies of the largest float below 2^-100 with a 24-bit significand
    of all ones, then of the same negated: each lane column's low word carries
    into its high word every 257th add, and the chunks cancel exactly."""
    v = np.uint32((27 << 23) | 0x7FFFFF)
    x = np.full(1 << 25, v, dtype=np.uint32)
    assert gpu32(x) == c_oracle.sum_f32_bits(x)
    y = np.concatenate([x, x | np.uint32(0x80000000)])
    assert gpu32(y) == 0


def test_method_values_rejected():
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    d = torch.zeros(4, dtype=torch.float32, device="cuda")
    for bad in (-1, 3):
        with pytest.raises(xsum.XsError) as e:
            xsum.xs_sum_f32_method_async(d, 4, out, bad)
        assert e.value.status == xsum.XS_ERR_INVALID_VALUE


@pytest.mark.parametrize("every", [3, 29, 1001])
def test_rare_terms_between_largest_slot_adds(every):
    """Same-sign floats at the top of a slot (e & 31 == 31: the largest adds,
    so slots approach their bound between propagations) with zeros and
    subnormals spread through them: groups holding one are taken back and
    re-added."""
    n = 4_000_037
    rng = np.random.default_rng(every)
    x = (np.uint32(223) << np.uint32(23)) | rng.integers(0, 1 << 23, n, dtype=np.uint32)
    sel = np.arange(every // 2, n, every)
    rare = np.array([0, 0x80000000, 1, 0x807FFFFF, 0x00400000], dtype=np.uint32)
    x[sel] = rare[rng.integers(0, rare.size, sel.size)]
    for mis in (0, 1, 3):
        assert gpu32(x, mis) == c_oracle.sum_f32_bits(x)
    x[n // 2] = 0xFF800000
    assert gpu32(x) == 0xFF800000
