"""GPU parity of the correctly rounded exact mean (and division of an
accumulator by any positive integer) against the oracle, bit for bit."""

import numpy as np
import pytest

import workloads as W
from oracle import c_oracle
from oracle import xsum_oracle as xo
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, f2b, out_slot, to_device

pytestmark = pytest.mark.gpu


def gpu_mean(bits, misalign=0):
    d = to_device(bits, misalign)
    out = out_slot()
    xsum.xs_mean_async(d, d.numel(), out)
    return int(bits_of(out)[0])


def test_worked_example():
    assert gpu_mean(W.f64_to_bits([1e15, -1e15, 0.1])) == f2b(0.1 / 3)


def test_cfg0_and_side_cases():
    x = W.f64_to_bits(W.cfg0_cancel(0))
    assert gpu_mean(x) == c_oracle.mean_bits(x)
    for _, vals in W.cfg2d_side_cases():
        b = W.f64_to_bits(np.array(vals, dtype=np.float64))
        for mis in (0, 1):
            assert gpu_mean(b, mis) == xo.mean_bits(b.tolist()), vals


@pytest.mark.parametrize("n", [1, 2, 3, 33, 4097, 100_003, 2_000_001])
def test_sizes(n):
    for x in (W.cfg2a_full_range(n, 0, n), W.cfg1_band(n, 0, n, -1074 + 52, -1000),
              W.cfg1_band(n + 1, 0, n)):
        assert gpu_mean(x) == c_oracle.mean_bits(x)


def test_tiny_and_subnormal_means():
    for b in ([1, 0], [3, 0], [1, 0, 0], [5, 0, 0, 0], [0x8000000000000003, 0]):
        arr = np.array(b, dtype=np.uint64)
        assert gpu_mean(arr) == xo.mean_bits(b)


def test_mean_never_overflows():
    dmax = 1.7976931348623157e308
    x = np.full(1_000_000, f2b(dmax), dtype=np.uint64)
    assert gpu_mean(x) == f2b(dmax)


def test_empty_mean_is_nan():
    out = out_slot()
    xsum.xs_mean_async(0, 0, out)
    assert int(bits_of(out)[0]) == 0x7FF8000000000000


def test_full_cfg1_mean():
    x = W.cfg1_band(0, 0, 10 ** 8)
    assert gpu_mean(x) == c_oracle.mean_bits(x)


def test_accumulator_division_by_any_divisor():
    x = W.cfg2a_paired(8, 0, 1_500_001)
    d = to_device(x)
    h = xsum.xs_acc_create()
    xsum.xs_acc_add(h, d[:700_000], 700_000)
    xsum.xs_acc_add(h, d[700_000:], x.size - 700_000)
    st = xo.state_of_bits(x.tolist())
    out = out_slot()
    for D in [1, 2, 3, x.size, 1000003, (1 << 32) + 1, (1 << 40) + 3, (1 << 63) - 25]:
        xsum.xs_acc_round_div(h, D, out)
        assert int(bits_of(out)[0]) == xo.finish_div(st, D), D
    xsum.xs_acc_destroy(h)


def _doubles_summing_to(S: int) -> list[int]:
    """Bit patterns of doubles whose exact sum is S * 2^-1074 (S >= 0): greedy
    53-bit pieces from the top, each exactly representable."""
    out = []
    while S:
        sh = max(0, S.bit_length() - 53)
        piece = (S >> sh) << sh
        out.append(f2b(float(__import__("fractions").Fraction(piece, 1 << 1074))))
        S -= piece
    return out


@pytest.mark.parametrize("d", [3, 5, 7, 64, 1000003])
@pytest.mark.parametrize("y", [1.0, 0.1, 3.0e300 / 7, 2.0 ** -1000])
def test_mean_ties_decided_by_the_lowest_chunk(d, y):
    """Sums with sum / n exactly halfway between two doubles (ties to even),
    and the same plus the smallest subnormal, which sits in chunk 0 far below
    the quotient's top: only the sticky part of the division breaks the tie."""
    Y = int(__import__("fractions").Fraction(y) * (1 << 1074))
    e = max(1, (Y.bit_length() - 53) + 1)  # ulp of y in units of 2^-1074 (normal y)
    U = 1 << (e - 1)
    for r in (0, 1):
        S = d * (2 * Y + U) // 2 + r if (d * U) % 2 == 0 else None
        if S is None:
            continue
        terms = _doubles_summing_to(S)
        if len(terms) > d:
            continue
        x = np.array(terms + [0] * (d - len(terms)), dtype=np.uint64)
        assert gpu_mean(x) == c_oracle.mean_bits(x), (d, y, r)
