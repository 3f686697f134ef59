"""The device generator reproduces the host generator bit for bit."""

import numpy as np
import pytest
import torch

import workloads as W
from workloads import devgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("start,count", [(0, 100_000), (123_456_789, 50_001)])
def test_device_generator_matches_host(start, count):
    t = torch.empty(count, dtype=torch.int64, device="cuda")
    devgen.band(t, 0, start)
    assert np.array_equal(t.cpu().numpy().view(np.uint64), W.cfg1_band(0, start, count))
    devgen.band(t, 3, start, -30, 30)
    assert np.array_equal(t.cpu().numpy().view(np.uint64), W.cfg3_values(3, start, count))
    devgen.full_range(t, 1, start)
    assert np.array_equal(t.cpu().numpy().view(np.uint64), W.cfg2a_full_range(1, start, count))
    devgen.paired(t, 2, start % (1 << 28))
    assert np.array_equal(t.cpu().numpy().view(np.uint64), W.cfg2a_paired(2, start % (1 << 28), count))
    devgen.cancel(t, 2, start % (1 << 28))
    assert np.array_equal(t.cpu().numpy().view(np.uint64),
                          W.cfg2b_cancel_1e300(2, start % (1 << 28), count))
