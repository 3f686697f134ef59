"""xs_sum_noalloc: the exact sum for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc: applications and frameworks
that manage all device memory through their own pool and budget, latency-bound
loops, processes whose device memory is already full. xs_sum_noalloc keeps its
only scratch (one 560-byte accumulator per device) in a static device array of
the library. This file is collected last, so a run that stops at the first
failure has run every other test first; it also passes alone in a fresh
process.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W
from oracle import c_oracle
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, out_slot, to_device

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def existing_entry_point_bits(d):
    out = out_slot()
    xsum.xs_sum_async(d, d.numel(), out, xsum.XS_METHOD_SMALL)
    return int(bits_of(out)[0])


def noalloc_bits(d, n=None):
    out = out_slot()
    xsum.xs_sum_noalloc(d, d.numel() if n is None else n, out)
    return int(bits_of(out)[0])


def test_noalloc_matches_oracle_and_xs_sum_async_on_two_calls_in_a_row():
    # first input carries Inf and a NaN, so a scratch left dirty by the first
    # call would spoil the second; the second is an ordinary large array
    first = W.cfg1_band(11, 0, 1_000_003).copy()
    first[[5, 77, 4000]] = [0x7FF0000000000000, 0x7FF8000000000099, 0xFFF0000000000000]
    second = W.cfg2a_paired(12, 0, 3_000_001)
    for x in (first, second):
        d = to_device(x)
        got = noalloc_bits(d)
        assert got == c_oracle.sum_bits(x)  # exact: tolerance 0
        assert got == existing_entry_point_bits(d)


def test_noalloc_edge_cases():
    """n = 0 (no kernel: the result slot is cleared to +0), an input whose
    first element is not 16-byte aligned (the kernel's head element), and an
    array past 2^25 values (where xs_sum_async picks another launch shape;
    xs_sum_noalloc keeps its one shape)."""
    out = out_slot()
    xsum.xs_sum_noalloc(out, 0, out)
    assert int(bits_of(out)[0]) == 0
    x = W.cfg0_cancel(3).view(np.uint64)
    d = to_device(x, misalign=1)
    assert noalloc_bits(d) == c_oracle.sum_bits(x)
    big = W.cfg1_band(13, 0, (1 << 25) + 3)
    d = to_device(big)
    assert noalloc_bits(d) == c_oracle.sum_bits(big)
    assert noalloc_bits(d) == existing_entry_point_bits(d)


_CHILD = r"""
import sys
import torch
sys.path.insert(0, sys.argv[1])
import workloads as W
from paper_1505_05571_gb300 import xsum
x = W.cfg1_band(14, 0, 2_000_001)
d = torch.from_numpy(x.view('int64')).cuda().view(torch.float64)
out = torch.empty(1, dtype=torch.float64, device='cuda')
torch.cuda.synchronize()
xsum.xs_sum_noalloc(d, d.numel(), out)  # first call: per-device set-up
xsum.xs_sum_noalloc(d, d.numel(), out)
torch.cuda.synchronize()
free_before, _ = torch.cuda.mem_get_info()
for _ in range(3):
    xsum.xs_sum_noalloc(d, d.numel(), out)
torch.cuda.synchronize()
free_after, _ = torch.cuda.mem_get_info()
print(int(out.view(torch.int64).item()) & ((1 << 64) - 1), free_before, free_after)
"""


def test_noalloc_in_a_fresh_process_allocates_nothing():
    """A process that calls only xs_sum_noalloc: free device memory is the same
    before and after three more calls, and the result is the oracle's."""
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    bits, free_before, free_after = (int(v) for v in r.stdout.split()[-3:])
    assert free_before == free_after
    assert bits == c_oracle.sum_bits(W.cfg1_band(14, 0, 2_000_001))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    # the library's own check, through a raw address (a tensor that small would
    # already be refused by the binding, since n values do not fit in it)
    out = out_slot()
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_sum_noalloc(out.data_ptr(), xsum.XS_NOALLOC_MAX_TERMS + 1, out)
    assert e.value.status == xsum.XS_ERR_INVALID_VALUE
    with pytest.raises(ValueError):
        xsum.xs_sum_noalloc(out, 2, out)
