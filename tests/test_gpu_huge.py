"""Inputs past 2^31 and 2^32 elements (17-34 GB on the device): 64-bit index
arithmetic in every kernel, and the mean's division by n >= 2^32. Expected
values come from closed forms evaluated with the oracle's integer rounding."""

import struct

import numpy as np
import pytest
import torch

from oracle import xsum_oracle as xo
from oracle import xsum_oracle32 as xo32
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, f2b, out_slot

pytestmark = pytest.mark.gpu


def K(v: float) -> int:
    """v as an exact signed integer multiple of 2^-1074."""
    b = f2b(v)
    k = xo.scaled_integer((b >> 52) & 0x7FF, b & ((1 << 52) - 1))
    return -k if b >> 63 else k


def rne(S: int) -> int:
    return xo.round_rne(S)


def free_bytes():
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("N", [(1 << 31) + 5, (1 << 32) + 3])
def test_sum_mean_and_segments_past_32_bit_indices(N):
    if free_bytes() < 8 * N + (4 << 30):
        pytest.skip("not enough device memory")
    v = 0.1
    d = torch.full((N,), v, dtype=torch.float64, device="cuda")
    out = out_slot()
    xsum.xs_sum_async(d, N, out)
    assert int(bits_of(out)[0]) == f2b(N * v)  # one IEEE multiply = RNE of the exact N v
    # terms at both ends and across the 2^31 boundary
    d[0] = 1e300
    d[N - 1] = -1e300
    d[1 << 31] = 3.0
    S = (N - 3) * K(v) + K(3.0)
    xsum.xs_sum_async(d, N, out)
    assert int(bits_of(out)[0]) == rne(S)
    xsum.xs_mean_async(d, N, out)
    assert int(bits_of(out)[0]) == xo.round_ratio(S, N)
    # two segments split just past 2^31
    cut = (1 << 31) + 1
    off = torch.tensor([0, cut, N], dtype=torch.int64, device="cuda")
    so = torch.empty(2, dtype=torch.float64, device="cuda")
    xsum.xs_sum_segments(d, off, 2, so)
    got = bits_of(so)
    S0 = K(1e300) + (cut - 2) * K(v) + K(3.0)  # d[0], d[1 .. 2^31 - 1], d[2^31]
    S1 = (N - cut - 1) * K(v) - K(1e300)
    assert int(got[0]) == rne(S0)
    assert int(got[1]) == rne(S1)
    del d


def test_binary32_sum_past_2_to_32_floats():
    N = (1 << 32) + 7
    if free_bytes() < 4 * N + (4 << 30):
        pytest.skip("not enough device memory")
    f = torch.full((N,), 0.1, dtype=torch.float32, device="cuda")
    o = torch.empty(1, dtype=torch.float32, device="cuda")
    xsum.xs_sum_f32_async(f, N, o)
    b = struct.unpack("<I", struct.pack("<f", 0.1))[0]
    k32 = ((1 << 23) + (b & 0x7FFFFF)) << (((b >> 23) & 0xFF) - 1)  # units of 2^-149
    got = int(o.view(torch.int32).cpu().numpy().view(np.uint32)[0])
    assert got == xo32.round_rne32(N * k32)
    del f
