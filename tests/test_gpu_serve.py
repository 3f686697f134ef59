"""Serving loop: continuous batching with device-resident session accumulators.

Each result must be the same bits alone and in the mix (and the oracle's):
exact sums do not depend on batching, order, or on how partial
superaccumulators are grouped (Discussion).
"""

import threading

import numpy as np
import pytest
import torch

import workloads as W
from oracle import c_oracle
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, f2b, out_slot, to_device

pytestmark = pytest.mark.gpu


def alone_sum(d, lo, hi):
    out = out_slot()
    xsum.xs_sum_async(d[lo:hi], hi - lo, out)
    return int(bits_of(out)[0])


def alone_session(d, ranges):
    h = xsum.xs_acc_create()
    for lo, hi in ranges:
        xsum.xs_acc_add(h, d[lo:hi], hi - lo)
    out = out_slot()
    xsum.xs_acc_round(h, out)
    xsum.xs_acc_destroy(h)
    return int(bits_of(out)[0])


def make_pool():
    n = 6_000_000
    x = W.cfg2a_paired(21, 0, n).copy()
    rng = np.random.default_rng(3)
    sel = rng.integers(0, n, 30)
    x[sel] = np.array([0x7FF0000000000000, 0x8000000000000000, 0x7FF8000000000011],
                      dtype=np.uint64)[rng.integers(0, 3, 30)]
    return x, to_device(x)


def random_range(rng, n_pool, big=False):
    m = int(np.exp(rng.uniform(0, np.log(2_000_000 if big else 200_000))))
    lo = int(rng.integers(0, n_pool - m))
    return lo, lo + m


# requests of at least long_min values are summed in block-wide tiles of
# long_tile values with a large superaccumulator; the others by one-warp groups
LONG_OPTS = [{}, {"long_min": 5000, "long_tile": 1024}, {"long_min": 1, "long_tile": 3001}]


@pytest.mark.parametrize("long_opts", LONG_OPTS, ids=[str(o) for o in LONG_OPTS])
def test_mix_matches_alone_and_oracle(long_opts):
    x, d = make_pool()
    server = xsum.xs_server_create(budget_bytes=64 << 20, streams=3, max_batch=64, tile_elems=1 << 16,
                                   **long_opts)
    rng = np.random.default_rng(7)
    plan = []  # (kind, ranges)
    for k in range(120):
        if rng.random() < 0.5:
            plan.append(("one", [random_range(rng, x.size, big=k % 10 == 0)]))
        else:
            g = int(rng.geometric(0.25))
            plan.append(("sess", [random_range(rng, x.size) for _ in range(g)]))
    ids = [None] * len(plan)

    def submitter(part):
        for k in part:
            kind, ranges = plan[k]
            if kind == "one":
                lo, hi = ranges[0]
                ids[k] = xsum.xs_server_submit(server, d[lo:hi], hi - lo)
            else:
                sid = xsum.xs_server_open_session(server)
                last = None
                for j, (lo, hi) in enumerate(ranges):
                    fl = xsum.XS_REQ_FINISH if j == len(ranges) - 1 else 0
                    last = xsum.xs_server_submit(server, d[lo:hi], hi - lo, session=sid, flags=fl)
                ids[k] = last

    threads = [threading.Thread(target=submitter, args=(list(range(i, len(plan), 2)),))
               for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    results = [xsum.xs_server_wait(server, rid, 60_000_000_000) for rid in ids]
    stats = xsum.xs_server_stats_get(server)
    xsum.xs_server_destroy(server)
    assert stats["completed"] == stats["submitted"]
    assert stats["batches"] < stats["submitted"]  # requests were batched
    for (kind, ranges), r in zip(plan, results):
        assert r["status"] == 0
        got = f2b(r["value"])
        if kind == "one":
            lo, hi = ranges[0]
            assert got == alone_sum(d, lo, hi)
            expect = c_oracle.sum_bits(x[lo:hi])
        else:
            assert got == alone_session(d, ranges)
            expect = c_oracle.sum_bits(np.concatenate([x[lo:hi] for lo, hi in ranges]))
        assert got == expect
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_launch_ns"] <= r["t_done_ns"]


def test_empty_and_tiny_requests():
    server = xsum.xs_server_create(streams=2)
    d = torch.tensor([1e15, -1e15, 0.1, -0.0], dtype=torch.float64, device="cuda")
    r0 = xsum.xs_server_submit(server, d, 0)
    r1 = xsum.xs_server_submit(server, d, 3)
    r2 = xsum.xs_server_submit(server, d[3:], 1)
    sid = xsum.xs_server_open_session(server)
    xsum.xs_server_submit(server, d, 1, session=sid)
    xsum.xs_server_submit(server, d[1:], 0, session=sid)
    r3 = xsum.xs_server_submit(server, d[1:], 2, session=sid, flags=xsum.XS_REQ_FINISH)
    vals = [xsum.xs_server_wait(server, r)["value"] for r in (r0, r1, r2, r3)]
    xsum.xs_server_destroy(server)
    assert f2b(vals[0]) == 0 and vals[1] == 0.1
    assert f2b(vals[2]) == 0x8000000000000000 and vals[3] == 0.1


def test_budget_and_misuse_errors():
    server = xsum.xs_server_create(budget_bytes=1 << 20, max_sessions=2)
    d = torch.zeros(1 << 18, dtype=torch.float64, device="cuda")
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_server_submit(server, d, 1 << 18)  # 2 MiB > 1 MiB budget
    assert e.value.status == xsum.XS_ERR_BUDGET
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_server_submit(server, torch.zeros(4, dtype=torch.float64), 4)  # host memory
    assert e.value.status == xsum.XS_ERR_INVALID_POINTER
    s1 = xsum.xs_server_open_session(server)
    xsum.xs_server_open_session(server)
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_server_open_session(server)  # no slot left
    assert e.value.status == xsum.XS_ERR_BUDGET
    r = xsum.xs_server_submit(server, d, 10, session=s1, flags=xsum.XS_REQ_FINISH)
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_server_submit(server, d, 10, session=s1)  # finished session
    assert e.value.status == xsum.XS_ERR_INVALID_VALUE
    assert xsum.xs_server_wait(server, r)["status"] == 0
    xsum.xs_server_destroy(server)


def test_wait_times_out_on_the_host():
    x = W.cfg1_band(2, 0, 50_000_000)
    d = to_device(x)
    server = xsum.xs_server_create(streams=1)
    rid = xsum.xs_server_submit(server, d, d.numel())
    rids = [xsum.xs_server_submit(server, d, d.numel()) for _ in range(4)]
    with pytest.raises(xsum.XsError) as e:
        xsum.xs_server_wait(server, rids[-1], 0)
    assert e.value.status == xsum.XS_ERR_TIMEOUT
    for r in [rid] + rids:
        assert f2b(xsum.xs_server_wait(server, r)["value"]) == c_oracle.sum_bits(x)
    xsum.xs_server_destroy(server)


@pytest.mark.parametrize("tile,long_tile", [(64, 0), (3000, 0), (1 << 20, 0), (0, 1024), (0, 3001),
                                            (0, 1 << 20), (0, 1 << 22)])
def test_tile_sizes_and_carries_inside_a_tile(tile, long_tile):
    """The smallest tile (64 values), an odd size, and tiles of 2^20 values,
    32,768 adds per thread of a one-warp group, where carries propagate inside
    the tile. Same-sign terms at the top of a chunk (the largest adds), a
    negative stretch (carries ripple as 2^32 - 1 chunks), zeros; a one-shot
    sum, a negative one and a two-part session."""
    rng = np.random.default_rng(tile)
    n = 3_000_017
    e = np.uint64(0x7DF)  # exponent 2015: chunk 62, shift 31
    x = (e << np.uint64(52)) | rng.integers(0, 1 << 52, n, dtype=np.uint64)
    x[1_000_000:2_000_000] |= np.uint64(1 << 63)
    x[rng.integers(0, n, 5000)] = 0
    d = to_device(x)
    # long_tile: every request in block-wide tiles; a tile of 2^22 such terms
    # carries out of a chunk's high word about 2^10 times
    server = xsum.xs_server_create(streams=2, tile_elems=tile, long_min=1 if long_tile else 1 << 30,
                                   long_tile=long_tile)
    r_all = xsum.xs_server_submit(server, d, n)
    r_neg = xsum.xs_server_submit(server, d[1_000_000:2_000_000], 1_000_000)
    sid = xsum.xs_server_open_session(server)
    xsum.xs_server_submit(server, d[:1_500_000], 1_500_000, session=sid)
    r_s = xsum.xs_server_submit(server, d[1_500_000:], n - 1_500_000, session=sid,
                                flags=xsum.XS_REQ_FINISH)
    got = [f2b(xsum.xs_server_wait(server, r, 60_000_000_000)["value"]) for r in (r_all, r_neg, r_s)]
    xsum.xs_server_destroy(server)
    full = c_oracle.sum_bits(x)
    assert got == [full, c_oracle.sum_bits(x[1_000_000:2_000_000]), full]


def test_tile_size_limits():
    for bad in (-5, 32, 63, 1 << 27):
        with pytest.raises(xsum.XsError) as e:
            xsum.xs_server_create(tile_elems=bad)
        assert e.value.status == xsum.XS_ERR_INVALID_VALUE
    for bad in ({"long_tile": 1000}, {"long_tile": 1 << 27}, {"long_min": -1}):
        with pytest.raises(xsum.XsError) as e:
            xsum.xs_server_create(**bad)
        assert e.value.status == xsum.XS_ERR_INVALID_VALUE


def test_serial_replay_matches_oracle():
    """The serial baseline (one request at a time, from a C loop): one-shot sums
    and sessions interleaved in the trace, each result the oracle's bits."""
    x, d = make_pool()
    base = d.data_ptr()
    rng = np.random.default_rng(11)
    items, expect = [], {}
    for k in range(40):
        if rng.random() < 0.5:
            lo, hi = random_range(rng, x.size)
            items.append((0, 0, base + 8 * lo, hi - lo, 0))
            expect[len(items) - 1] = c_oracle.sum_bits(x[lo:hi])
        else:
            ranges = [random_range(rng, x.size) for _ in range(int(rng.geometric(0.3)))]
            for j, (lo, hi) in enumerate(ranges):
                fin = j == len(ranges) - 1
                items.append((0, k + 1, base + 8 * lo, hi - lo, xsum.XS_REQ_FINISH if fin else 0))
            expect[len(items) - 1] = c_oracle.sum_bits(np.concatenate([x[lo:hi] for lo, hi in ranges]))
    items.append((0, 0, base, 0, 0))  # an empty one-shot sum
    expect[len(items) - 1] = 0
    vals, done = xsum.xs_serial_replay(items)
    assert all(b >= a for a, b in zip(done, done[1:]))
    for k, e in expect.items():
        assert f2b(vals[k]) == e, k
