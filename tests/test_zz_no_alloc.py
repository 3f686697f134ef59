"""xs_sum_noalloc: the exact sum for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc: applications and frameworks
that manage all device memory through their own pool and budget, latency-bound
loops, processes whose device memory is already full. xs_sum_noalloc keeps its
only scratch (one 560-byte accumulator per device) in a static device array of
the library. This file is collected last, so a run that stops at the first
failure has run every other test first; it also passes alone in a fresh
process.
"""

import pytest

import workloads as W
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, out_slot, to_device

pytestmark = pytest.mark.gpu


def existing_entry_point_bits(d):
    out = out_slot()
    xsum.xs_sum_async(d, d.numel(), out, xsum.XS_METHOD_SMALL)
    return int(bits_of(out)[0])


def test_noalloc_matches_xs_sum_async_on_two_calls_in_a_row():
    # first input carries Inf and a NaN, so a scratch left dirty by the first
    # call would spoil the second; the second is an ordinary large array
    first = W.cfg1_band(11, 0, 1_000_003).copy()
    first[[5, 77, 4000]] = [0x7FF0000000000000, 0x7FF8000000000099, 0xFFF0000000000000]
    second = W.cfg2a_paired(12, 0, 3_000_001)
    for x in (first, second):
        d = to_device(x)
        out = out_slot()
        xsum.xs_sum_noalloc(d, d.numel(), out)
        got = int(bits_of(out)[0])
        assert got == existing_entry_point_bits(d)  # exact: tolerance 0


def test_noalloc_rejects_sizes_beyond_its_maximum():
    out = out_slot()
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_sum_noalloc(out, xsum.XS_NOALLOC_MAX_TERMS + 1, out)
    assert e.value.status == xsum.XS_ERR_INVALID_VALUE
