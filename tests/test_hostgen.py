"""The multithreaded host generator gives the numpy recipe's bits exactly, for
both exponent bands, at several start offsets and across thread boundaries."""

import numpy as np
import pytest

import workloads as W
from workloads import hostgen


@pytest.mark.parametrize("seed,start,count,lo,hi", [
    (0, 0, 1, -60, 60),
    (0, 0, 100_003, -60, 60),
    (0, 7_200_000_000, 50_001, -30, 30),   # far into the segmented workload
    (3, 123_456_789, 77_777, -30, 30),
    (5, (1 << 33) + 11, 4097, -1022, 1023),
])
def test_host_twin_matches_numpy(seed, start, count, lo, hi):
    got = hostgen.band(seed, start, count, lo, hi)
    assert got.dtype == np.uint64
    assert np.array_equal(got, W.cfg1_band(seed, start, count, lo, hi))


def test_host_twin_fills_a_prefix_of_a_larger_buffer():
    buf = np.full(1000, 0xDEADBEEF, dtype=np.uint64)
    got = hostgen.band(1, 10, 600, -30, 30, out=buf)
    assert got.size == 600
    assert np.array_equal(got, W.cfg3_values(1, 10, 600))
    assert np.all(buf[600:] == 0xDEADBEEF)
    assert hostgen.band(1, 10, 0).size == 0
