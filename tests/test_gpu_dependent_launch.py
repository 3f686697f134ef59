"""Back-to-back sums on one stream: the single-array kernels are launched with
programmatic stream serialization, so a sum may be scheduled while the one
before it finishes. A sum whose input holds the previous sum's result (written
by the previous grid's last block) must see that result, and sums that share
the stream's workspace accumulator must not mix."""

import pytest
import torch

import workloads as W
from oracle import c_oracle, products
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_y", [2, 1001, 3_000_001])
def test_next_sum_reads_the_previous_result(n_y):
    x = to_device(W.cfg1_band(21, 0, 2_000_001))
    y = to_device(W.cfg1_band(22, 0, n_y))
    y[0] = float("nan")  # overwritten by the first sum before the second may read it
    chain = torch.empty(8, dtype=torch.float64, device="cuda")
    # sum(x) -> y[0]; sum(y) -> chain[0]; mean(y) -> chain[1]; dot(y, y) -> chain[2]; ...
    xsum.xs_sum_async(x, x.numel(), y[0:1])
    xsum.xs_sum_async(y, n_y, chain[0:1])
    xsum.xs_mean_async(y, n_y, chain[1:2])
    xsum.xs_dot_async(y, y, n_y, chain[2:3])
    xsum.xs_sum_async(chain[0:3], 3, chain[3:4])
    torch.cuda.synchronize()
    xb = bits_of(x)
    yb = bits_of(y)
    assert int(yb[0]) == c_oracle.sum_bits(xb)
    cb = bits_of(chain)
    assert int(cb[0]) == c_oracle.sum_bits(yb)
    assert int(cb[1]) == c_oracle.mean_bits(yb)
    assert int(cb[2]) == products.dot_bits(yb, yb)
    assert int(cb[3]) == c_oracle.sum_bits(cb[:3])


def test_many_back_to_back_sums_share_the_workspace():
    """40 sums of different arrays queued without a synchronisation in between
    (each grid may start before the previous has reset the accumulator)."""
    arrays = [to_device(W.cfg2a_paired(30 + k, 0, 100_003 + 7919 * k)) for k in range(8)]
    out = torch.empty(40, dtype=torch.float64, device="cuda")
    for j in range(40):
        a = arrays[j % 8]
        xsum.xs_sum_async(a, a.numel(), out[j:j + 1])
    torch.cuda.synchronize()
    got = bits_of(out)
    expect = [c_oracle.sum_bits(bits_of(a)) for a in arrays]
    for j in range(40):
        assert int(got[j]) == expect[j % 8], j
