"""Every head length before the first 256-byte boundary (0..31 doubles, 0..63
floats): the streamed body starts on that boundary and the elements before it
are added apart, so each start offset must give the oracle's bits, for the
single-array methods, the dot product, the binary32 sum, segments and served
requests. Offsets are taken from one 256-byte-aligned buffer."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import c_oracle, products
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, out_slot

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 31, 32, 33, 63, 1000, 100_003]


@pytest.fixture(scope="module")
def pool():
    x = W.cfg2a_paired(41, 0, 200_000 + 64)
    d = torch.empty(x.size + 64, dtype=torch.int64, device="cuda")
    base = (-d.data_ptr() // 8) % 32  # first element on a 256-byte boundary
    d = d[base:base + x.size]
    d.copy_(torch.from_numpy(x.view(np.int64)))
    assert d.data_ptr() % 256 == 0
    return x, d.view(torch.float64)


@pytest.mark.parametrize("shift", list(range(33)))
def test_single_array_every_head_length(pool, shift):
    x, d = pool
    out = out_slot()
    for n in SIZES:
        seg = x[shift:shift + n]
        expect = c_oracle.sum_bits(seg)
        for m, b, u in ((xsum.XS_METHOD_SMALL, 384, 4), (xsum.XS_METHOD_SMALL, 384, 6),
                        (xsum.XS_METHOD_LARGE, 768, 4), (xsum.XS_METHOD_LARGE, 512, 4)):
            xsum.xs_sum_async_config(d[shift:], n, out, m, b, u, 0)
            assert int(bits_of(out)[0]) == expect, (shift, n, m, b, u)


@pytest.mark.parametrize("shift", [0, 1, 7, 16, 31, 32])
def test_dot_every_head_length(pool, shift):
    x, d = pool
    out = out_slot()
    for n in SIZES:
        for yshift in (0, 1, 5):
            xs, ys = x[shift:shift + n], x[1000 + yshift:1000 + yshift + n]
            expect = products.dot_bits(xs, ys)
            for m in (xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE):
                xsum.xs_dot_method_async(d[shift:], d[1000 + yshift:], n, out, m)
                assert int(bits_of(out)[0]) == expect, (shift, yshift, n, m)


@pytest.mark.parametrize("shift", [0, 1, 2, 3, 17, 31, 32, 33, 62, 63, 64])
def test_binary32_every_head_length(shift):
    rng = np.random.default_rng(shift)
    m = 100_000 + 128
    h = ((rng.integers(67, 187, m, dtype=np.uint32) << np.uint32(23))
         | rng.integers(0, 1 << 23, m, dtype=np.uint32)
         | (rng.integers(0, 2, m, dtype=np.uint32) << np.uint32(31)))
    t = torch.empty(m + 64, dtype=torch.int32, device="cuda")
    base = (-t.data_ptr() // 4) % 64
    t = t[base:base + m]
    t.copy_(torch.from_numpy(h.view(np.int32)))
    assert t.data_ptr() % 256 == 0
    o32 = torch.empty(1, dtype=torch.float32, device="cuda")
    for n in (1, 3, 63, 64, 65, 99_999):
        for m in (xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE):
            xsum.xs_sum_f32_method_async(t[shift:].view(torch.float32), n, o32, m)
            got = int(o32.view(torch.int32).cpu().numpy().view(np.uint32)[0])
            assert got == c_oracle.sum_f32_bits(h[shift:shift + n]), (shift, n, m)


def test_segments_and_served_requests_at_every_offset(pool):
    """Segments of lengths 1..300 laid end to end start at every offset mod
    256 bytes; the same ranges as served requests, both through the one-warp
    tiles and through block-wide tiles of long requests."""
    x, d = pool
    lengths = np.array([(k * 37) % 300 + 1 for k in range(600)], dtype=np.int64)
    off = W.cfg3_offsets(lengths)
    expect = c_oracle.segment_sums_bits(x, off)
    od = torch.from_numpy(off).cuda()
    out = torch.empty(lengths.size, dtype=torch.float64, device="cuda")
    for opts in (None, {"block": 128, "unroll": 8, "tile_elems": 256, "short_max": 0},
                 {"block": 32, "unroll": 8, "tile_elems": 100, "short_max": 16}):
        p = xsum.xs_seg_plan_create(d, od, lengths.size, out, opts)
        try:
            xsum.xs_seg_plan_launch(p)
            torch.cuda.synchronize()
        finally:
            xsum.xs_seg_plan_destroy(p)
        assert np.array_equal(bits_of(out), expect), opts
    for long_opts in ({}, {"long_min": 1, "long_tile": 1024}):
        srv = xsum.xs_server_create(streams=2, tile_elems=64, **long_opts)
        try:
            ids = [xsum.xs_server_submit(srv, d[int(off[k]):], int(lengths[k])) for k in range(lengths.size)]
            vals = [xsum.xs_server_wait(srv, r, 60_000_000_000)["value"] for r in ids]
        finally:
            xsum.xs_server_destroy(srv)
        got = np.array(vals, dtype=np.float64).view(np.uint64)
        assert np.array_equal(got, expect), long_opts
