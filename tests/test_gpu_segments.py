"""Batched segmented exact sums (CSR) against the oracle, per segment, bit for bit."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import c_oracle
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, to_device
from workloads import devgen, hostgen

pytestmark = pytest.mark.gpu

OPTS = [
    None,
    {"block": 128, "unroll": 4, "tile_elems": 1 << 12, "short_max": 64},
    {"block": 192, "unroll": 4, "tile_elems": 1 << 16, "short_max": 1024},
    {"block": 256, "unroll": 4, "tile_elems": 1 << 13, "short_max": 4096},
    {"block": 384, "unroll": 4, "tile_elems": 1 << 18, "short_max": 16384},
    {"block": 192, "unroll": 8, "tile_elems": 3000, "short_max": 0},
    {"block": 128, "unroll": 8, "tile_elems": 1 << 14, "short_max": 256},
    {"block": 64, "unroll": 8, "tile_elems": 1 << 15, "short_max": 4096},
    {"block": 32, "unroll": 8, "tile_elems": 5000, "short_max": 128},
    {"block": 32, "unroll": 8, "tile_elems": 1 << 17, "short_max": 0},
]


def mixed_lengths(seed, nseg):
    rng = np.random.default_rng(seed)
    lengths = W.cfg3_lengths(seed, nseg, 200_000)
    special = np.array([0, 1, 2, 3, 31, 32, 33, 64, 65, 4096, 4097, 8191, 8193, 12289], dtype=np.int64)
    pos = rng.integers(0, nseg, special.size)
    lengths[pos] = special
    return lengths


def run_plan(vals_dev, off_dev, nseg, opts, graph=True):
    out = torch.full((nseg,), float("nan"), dtype=torch.float64, device="cuda")
    p = xsum.xs_seg_plan_create(vals_dev, off_dev, nseg, out, opts)
    try:
        for _ in range(2):  # repeated launches reuse the self-resetting work space
            out.fill_(float("nan"))
            if graph:
                xsum.xs_seg_plan_launch(p)
            else:
                xsum.xs_seg_plan_launch_direct(p)
        torch.cuda.synchronize()
    finally:
        xsum.xs_seg_plan_destroy(p)
    return bits_of(out)


@pytest.mark.parametrize("opts", OPTS, ids=[str(o) for o in OPTS])
def test_segments_mixed(opts):
    nseg = 3000
    lengths = mixed_lengths(1, nseg)
    off = W.cfg3_offsets(lengths)
    vals = W.cfg2a_paired(5, 0, int(off[-1]))
    specials = np.array([0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000077,
                         0x8000000000000000], dtype=np.uint64)
    rng = np.random.default_rng(2)
    sel = rng.integers(0, vals.size, 40)
    vals[sel] = specials[rng.integers(0, 4, sel.size)]
    # a segment of only -0 and one of +0, -0
    z0 = int(np.argmax(lengths == 3))
    vals[off[z0]:off[z0 + 1]] = 0x8000000000000000
    expect = c_oracle.segment_sums_bits(vals, off)
    vd = to_device(vals)
    od = torch.from_numpy(off).cuda()
    got = run_plan(vd, od, nseg, opts)
    bad = np.nonzero(got != expect)[0]
    assert bad.size == 0, [(int(k), int(lengths[k]), hex(got[k]), hex(expect[k])) for k in bad[:5]]
    got2 = run_plan(vd, od, nseg, opts, graph=False)
    assert np.array_equal(got2, expect)


def test_segments_unaligned_values_and_convenience_api():
    nseg = 500
    lengths = mixed_lengths(3, nseg)
    off = W.cfg3_offsets(lengths)
    vals = W.cfg3_values(3, 0, int(off[-1]))
    vd = to_device(vals, misalign=1)
    od = torch.from_numpy(off).cuda()
    out = torch.empty(nseg, dtype=torch.float64, device="cuda")
    xsum.xs_sum_segments(vd, od, nseg, out)
    xsum.xs_sum_segments(vd, od, nseg, out)  # cached plan, graph replay
    assert np.array_equal(bits_of(out), c_oracle.segment_sums_bits(vals, off))


def test_segments_repeats_closed_form():
    """Long segments of one repeated value: fl(N v) per segment, across tiles."""
    vs = [0.1, 1.0 - 2.0 ** -53, 3 * 5e-324, -0.7]
    Ns = [1, 2, 4095, 4097, 300_001]
    lengths, vals, expect = [], [], []
    for v in vs:
        for N in Ns:
            lengths.append(N)
            vals.append(np.full(N, v))
            expect.append(np.array([v * N]).view(np.uint64)[0])
    off = W.cfg3_offsets(np.array(lengths, dtype=np.int64))
    vd = torch.from_numpy(np.concatenate(vals)).cuda()
    od = torch.from_numpy(off).cuda()
    got = run_plan(vd, od, len(lengths), {"block": 192, "unroll": 4, "tile_elems": 8192,
                                          "short_max": 1024})
    assert np.array_equal(got, np.array(expect, dtype=np.uint64))


def test_segments_autotune_then_default():
    nseg = 2000
    lengths = mixed_lengths(4, nseg)
    off = W.cfg3_offsets(lengths)
    vals = W.cfg3_values(4, 0, int(off[-1]))
    vd, od = to_device(vals), torch.from_numpy(off).cuda()
    out = torch.empty(nseg, dtype=torch.float64, device="cuda")
    best = xsum.xs_autotune_segments(vd, od, nseg, out, reps=2)
    assert best["us"] > 0
    got = run_plan(vd, od, nseg, None)
    assert np.array_equal(got, c_oracle.segment_sums_bits(vals, off))


def cfg3_oracle_all(off: np.ndarray, seed: int = 0, slice_values: int = 1 << 28) -> np.ndarray:
    """Oracle bits of every segment of the segmented workload: the host
    regenerates the values in slices of whole segments (about 2 GB each, on
    every host core) and the C oracle sums each slice's segments on OpenMP
    threads."""
    nseg = off.size - 1
    expect = np.empty(nseg, dtype=np.uint64)
    buf = np.empty(max(slice_values, int(np.diff(off).max())), dtype=np.uint64)
    s0 = 0
    while s0 < nseg:
        s1 = int(np.searchsorted(off, off[s0] + slice_values, side="right")) - 1
        s1 = min(max(s1, s0 + 1), nseg)
        lo, hi = int(off[s0]), int(off[s1])
        vals = hostgen.band(seed, lo, hi - lo, -30, 30, out=buf)
        expect[s0:s1] = c_oracle.segment_sums_bits(vals, off[s0:s1 + 1] - lo)
        s0 = s1
    return expect


def test_full_cfg3_every_segment():
    """100,000 segments, lengths log-uniform in [1, 1e6] (about 7.3e9 values,
    58 GB generated in HBM), autotuned options: every segment's sum equals the
    oracle's bit for bit."""
    nseg = 100_000
    lengths = W.cfg3_lengths(0, nseg, 10 ** 6)
    off = W.cfg3_offsets(lengths)
    total = int(off[-1])
    free, _ = torch.cuda.mem_get_info()
    if total * 8 > free - (8 << 30):
        pytest.skip(f"needs {total * 8 / 2**30:.1f} GiB free, have {free / 2**30:.1f}")
    vals = torch.empty(total, dtype=torch.int64, device="cuda")
    devgen.band(vals, 0, 0, -30, 30)
    od = torch.from_numpy(off).cuda()
    out = torch.empty(nseg, dtype=torch.float64, device="cuda")
    vd = vals.view(torch.float64)
    got = {}
    xsum.xs_sum_segments(vd, od, nseg, out)  # default options
    got["default"] = bits_of(out)
    xsum.xs_autotune_segments(vd, od, nseg, out, reps=1)
    out.fill_(float("nan"))
    p = xsum.xs_seg_plan_create(vd, od, nseg, out, None)  # the tuned options
    try:
        xsum.xs_seg_plan_launch(p)
        torch.cuda.synchronize()
    finally:
        xsum.xs_seg_plan_destroy(p)
    got["tuned"] = bits_of(out)
    del vals, vd
    torch.cuda.empty_cache()
    expect = cfg3_oracle_all(off)
    for name, g in got.items():
        bad = np.nonzero(g != expect)[0]
        assert bad.size == 0, (name, bad.size, [(int(k), int(lengths[k])) for k in bad[:5]])


@pytest.mark.parametrize("tile", [1 << 20, 1 << 22, 3_000_001])
def test_tiles_longer_than_the_carry_interval(tile):
    """Tiles of up to 4 Mi values per 128-thread group (about 32,000 adds per
    thread): carries propagate inside the tile, and the merge window then runs
    to the top chunk. Same-sign terms at the top of a chunk (the largest
    adds), a negative segment (carries ripple as 2^32 - 1 chunks), zeros."""
    rng = np.random.default_rng(tile)
    lengths = np.array([3_000_017, 5, 4_200_000, 1, 2_500_001], dtype=np.int64)
    off = W.cfg3_offsets(lengths)
    n = int(off[-1])
    e = np.uint64(0x7DF)  # exponent 2015: chunk 62, shift 31
    vals = (e << np.uint64(52)) | rng.integers(0, 1 << 52, n, dtype=np.uint64)
    vals[off[2]:off[3]] |= np.uint64(1 << 63)  # the third segment negative
    vals[rng.integers(0, n, 5000)] = 0
    expect = c_oracle.segment_sums_bits(vals, off)
    vd = to_device(vals)
    od = torch.from_numpy(off).cuda()
    for opts in ({"block": 128, "unroll": 8, "tile_elems": tile, "short_max": 64},
                 {"block": 192, "unroll": 4, "tile_elems": tile, "short_max": 0},
                 {"block": 128, "unroll": 8, "tile_elems": tile, "short_max": 64, "carry_tiles": 1},
                 {"block": 192, "unroll": 4, "tile_elems": tile, "short_max": 64, "carry_tiles": 37},
                 {"block": 32, "unroll": 8, "tile_elems": tile, "short_max": 64}):
        got = run_plan(vd, od, lengths.size, opts)
        assert np.array_equal(got, expect), (opts, [hex(int(g)) for g in got], [hex(int(x)) for x in expect])
    out = torch.empty(lengths.size, dtype=torch.float64, device="cuda")
    with pytest.raises(xsum.XsError) as e:  # longer than 2047 adds between propagations
        xsum.xs_seg_plan_create(vd, od, lengths.size, out, {"block": 128, "unroll": 8, "carry_tiles": 128})
    assert e.value.status == xsum.XS_ERR_INVALID_VALUE


@pytest.mark.parametrize("dist", ["band", "full_range", "paired", "specials"])
def test_tiny_segments_one_lane_each(dist):
    """Segments of 0..140 values: those of up to 128 are summed by one lane
    each and rounded side by side, the longer ones (and lanes whose chunk
    window is too wide) by the warp; every result against the oracle."""
    rng = np.random.default_rng(11)
    lengths = rng.integers(0, 141, 40_000).astype(np.int64)
    lengths[rng.integers(0, lengths.size, 500)] = rng.integers(0, 3, 500)  # many of 0, 1, 2
    off = W.cfg3_offsets(lengths)
    n = int(off[-1])
    if dist == "band":
        vals = W.cfg3_values(6, 0, n)
    elif dist == "full_range":
        vals = W.cfg2a_full_range(6, 0, n)
    elif dist == "paired":
        vals = W.cfg2a_paired(6, 0, n)
    else:
        vals = W.cfg3_values(7, 0, n)
        specials = np.array([0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000123,
                             0xFFF4000000000001, 0x8000000000000000, 0x0000000000000001,
                             0x800FFFFFFFFFFFFF, 0x7FEFFFFFFFFFFFFF], dtype=np.uint64)
        sel = rng.integers(0, n, n // 50)
        vals[sel] = specials[rng.integers(0, specials.size, sel.size)]
    expect = c_oracle.segment_sums_bits(vals, off)
    vd, od = to_device(vals), torch.from_numpy(off).cuda()
    for opts in (None, {"block": 32, "unroll": 8, "short_max": 100}, {"block": 384, "unroll": 4, "short_max": 4096}):
        got = run_plan(vd, od, lengths.size, opts)
        bad = np.nonzero(got != expect)[0]
        assert bad.size == 0, (opts, [(int(k), int(lengths[k]), hex(got[k]), hex(expect[k])) for k in bad[:5]])


def test_golden_boundary_cases_as_short_segments():
    """Every hand-derived boundary case (ties to even, sticky bits from
    2^-1074, overflow at the midpoint below 2^1024, subnormal results, signed
    zeros, Inf/NaN rules) as one short segment, repeated with padding zeros and
    with the terms scaled into other chunks: the one-thread rounding of small
    windows and the warp rounding must both give the expected bits."""
    from tests.test_oracle import GOLDEN_CASES
    segs, expect = [], []
    for name, bits, exp in GOLDEN_CASES:
        segs.append(list(bits))
        expect.append(exp)
        if bits:  # the same case followed by zeros (+0 keeps -0 results -0 only if all are -0)
            padded = list(bits) + [0x8000000000000000] * 40
            segs.append(padded)
            expect.append(c_oracle.sum_bits(np.array(padded, dtype=np.uint64)))
    # windows of every width near the 8-chunk limit: one term per chunk
    for width in range(1, 12):
        bits = [int(np.array([2.0 ** (32 * k - 300) * (1 + k / 7)], dtype=np.float64).view(np.uint64)[0])
                for k in range(width)]
        bits.append(int(np.array([-(2.0 ** -300)], dtype=np.float64).view(np.uint64)[0]))
        segs.append(bits)
        expect.append(c_oracle.sum_bits(np.array(bits, dtype=np.uint64)))
    lengths = np.array([len(x) for x in segs], dtype=np.int64)
    off = W.cfg3_offsets(lengths)
    flat = np.array([b for x in segs for b in x], dtype=np.uint64)
    vd = to_device(flat if flat.size else np.zeros(1, dtype=np.uint64))
    od = torch.from_numpy(off).cuda()
    for opts in ({"block": 128, "unroll": 8, "short_max": 4096}, {"block": 192, "unroll": 4, "short_max": 64}):
        got = run_plan(vd, od, lengths.size, opts)
        bad = [(k, hex(int(got[k])), hex(int(expect[k]))) for k in range(lengths.size) if int(got[k]) != int(expect[k])]
        assert not bad, (opts, bad[:5])


@pytest.mark.parametrize("block,unroll", [(32, 8), (128, 8)])
def test_offsets_rewritten_in_place_past_the_tile_table(block, unroll):
    """A plan replays over the offsets as they are at launch. Rewritten in place
    to many more tiles than the plan's tile table holds, the tiles find their
    segment by a binary search over the tile prefix sums (short segments, with
    no tiles, sit between long ones)."""
    nseg = 40
    small = np.full(nseg, 10, dtype=np.int64)
    big = W.cfg3_lengths(9, nseg, 200_000)
    big[::7] = 3
    off_small, off_big = W.cfg3_offsets(small), W.cfg3_offsets(big)
    vals = W.cfg3_values(9, 0, int(off_big[-1]))
    vd = to_device(vals)
    od = torch.from_numpy(off_small).cuda()
    out = torch.full((nseg,), float("nan"), dtype=torch.float64, device="cuda")
    p = xsum.xs_seg_plan_create(vd, od, nseg, out,
                                {"block": block, "unroll": unroll, "tile_elems": 4096, "short_max": 64})
    try:
        xsum.xs_seg_plan_launch(p)
        torch.cuda.synchronize()
        assert np.array_equal(bits_of(out), c_oracle.segment_sums_bits(vals, off_small))
        od.copy_(torch.from_numpy(off_big))
        out.fill_(float("nan"))
        xsum.xs_seg_plan_launch(p)
        torch.cuda.synchronize()
        assert np.array_equal(bits_of(out), c_oracle.segment_sums_bits(vals, off_big))
    finally:
        xsum.xs_seg_plan_destroy(p)


def test_one_launch_per_segment_baseline_matches_oracle():
    """The comparison baseline (one single-array launch per segment from a C
    loop, host offsets) gives the oracle's bits, empty segments included."""
    nseg = 700
    lengths = mixed_lengths(5, nseg)
    off = W.cfg3_offsets(lengths)
    vals = W.cfg3_values(5, 0, int(off[-1]))
    vd = to_device(vals, misalign=1)
    out = torch.full((nseg,), float("nan"), dtype=torch.float64, device="cuda")
    xsum.xs_sum_each_async(vd, off, nseg, out)
    assert np.array_equal(bits_of(out), c_oracle.segment_sums_bits(vals, off))
    bad = off.copy()
    bad[3], bad[4] = bad[4], bad[3]  # decreasing offsets: rejected on the host
    if bad[3] != bad[4]:
        with pytest.raises(xsum.XsError) as e:
            xsum.xs_sum_each_async(vd, bad, nseg, out)
        assert e.value.status == xsum.XS_ERR_INVALID_VALUE


def test_malformed_offsets_are_flagged_and_not_read():
    """Offsets that decrease (all inside the values, so nothing out of bounds
    is ever at stake) and a first offset other than 0: the launch flags the
    plan, each malformed segment holds the default NaN without being read,
    and every well-formed segment is still the oracle's sum."""
    vals = W.cfg3_values(8, 0, 100_000)
    vd = to_device(vals)
    cases = [
        np.array([0, 10, 5, 20_000, 20_000, 90_000, 30, 40], dtype=np.int64),  # two decreases
        np.array([7, 500, 70_000, 99_000], dtype=np.int64),                      # first offset not 0
        np.array([0, 60_000, 100_000], dtype=np.int64),                          # well formed
    ]
    for off in cases:
        nseg = off.size - 1
        od = torch.from_numpy(off).cuda()
        for opts in (None, {"block": 128, "unroll": 8, "tile_elems": 4096, "short_max": 64}):
            out = torch.zeros(nseg, dtype=torch.float64, device="cuda")
            p = xsum.xs_seg_plan_create(vd, od, nseg, out, opts)
            try:
                xsum.xs_seg_plan_launch(p)
                bad = [k for k in range(nseg) if off[k + 1] < off[k] or off[k] < 0]
                if bad or off[0] != 0:
                    with pytest.raises(xsum.XsError) as e:
                        xsum.xs_seg_plan_check(p)
                    assert e.value.status == xsum.XS_ERR_INVALID_VALUE
                else:
                    xsum.xs_seg_plan_check(p)
                got = bits_of(out)
                for k in range(nseg):
                    if k in bad:
                        assert got[k] == 0x7FF8000000000000, k
                    else:
                        assert got[k] == c_oracle.sum_bits(vals[off[k]:off[k + 1]]), k
                # the status is per launch: after the offsets are fixed in place it clears
                if bad:
                    good = np.maximum.accumulate(off) - off[0]
                    od.copy_(torch.from_numpy(good))
                    xsum.xs_seg_plan_launch(p)
                    xsum.xs_seg_plan_check(p)
                    od.copy_(torch.from_numpy(off))
            finally:
                xsum.xs_seg_plan_destroy(p)
