"""Allocation failures injected on the host (xs_debug_fail_allocation): every
entry point that allocates reports XS_ERR_OUT_OF_MEMORY, frees what it had
allocated before the failure (the library's live-allocation count is back
where it was), and the same call succeeds, with the oracle's bits, once
memory is available again. No GPU fault is involved: the failure is made on
the host before cudaMalloc is called."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import c_oracle
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, f2b, out_slot, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def disarm():
    yield
    xsum.xs_debug_fail_allocation(0)


def fail_each_allocation(call, max_allocs=16):
    """Runs call() with the k-th allocation failing, k = 1, 2, ..., until it
    succeeds; returns its result and the number of allocations it made."""
    for k in range(1, max_allocs + 1):
        live = xsum.xs_debug_live_allocations()
        xsum.xs_debug_fail_allocation(k)
        try:
            r = call()
        except xsum.XsError as e:
            assert e.status == xsum.XS_ERR_OUT_OF_MEMORY, (k, e)
            assert xsum.xs_debug_live_allocations() == live, k
            continue
        xsum.xs_debug_fail_allocation(0)
        return r, k - 1
    raise AssertionError("never succeeded")


@pytest.fixture()
def data():
    x = W.cfg1_band(31, 0, 300_001)
    return x, to_device(x)


def test_workspace_of_a_new_stream(data):
    x, d = data
    s = torch.cuda.Stream()
    out = out_slot()
    _, n = fail_each_allocation(lambda: xsum.xs_sum_async(d, d.numel(), out, 0, s))
    assert n == 2  # the accumulators and the mapped result slot
    s.synchronize()
    assert int(bits_of(out)[0]) == c_oracle.sum_bits(x)


def stream_with_workspace(d):
    """A new stream whose workspace (kept for later calls by design) exists."""
    s = torch.cuda.Stream()
    xsum.xs_sum_async(d, d.numel(), out_slot(), 0, s)
    s.synchronize()
    return s


def test_host_buffer_staging(data):
    x, d = data
    s = stream_with_workspace(d)
    h = torch.from_numpy(x.view(np.float64)).pin_memory()
    r, n = fail_each_allocation(lambda: xsum.xs_sum_host(h, h.numel(), s))
    assert n == 2  # the two staging slots
    assert f2b(r) == c_oracle.sum_bits(x)


def test_inexact_baseline_partials(data):
    _, d = data
    s = stream_with_workspace(d)
    out = out_slot()
    _, n = fail_each_allocation(lambda: xsum.xs_inexact_sum_async(d, d.numel(), out, s))
    assert n == 1


def test_accumulator_handle(data):
    x, d = data
    h, n = fail_each_allocation(lambda: xsum.xs_acc_create())
    assert n == 1
    try:
        xsum.xs_acc_add(h, d, d.numel())
        out = out_slot()
        xsum.xs_acc_round(h, out)
        assert int(bits_of(out)[0]) == c_oracle.sum_bits(x)
    finally:
        xsum.xs_acc_destroy(h)


def test_segmented_plan(data):
    x, d = data
    off = np.array([0, 5, 100_000, 100_000, 300_001], dtype=np.int64)
    od = torch.from_numpy(off).cuda()
    out = torch.empty(off.size - 1, dtype=torch.float64, device="cuda")
    p, n = fail_each_allocation(lambda: xsum.xs_seg_plan_create(d, od, off.size - 1, out))
    assert n == 1
    try:
        xsum.xs_seg_plan_launch(p)
        torch.cuda.synchronize()
        assert np.array_equal(bits_of(out), c_oracle.segment_sums_bits(x, off))
    finally:
        xsum.xs_seg_plan_destroy(p)


def test_server(data):
    x, d = data
    srv, n = fail_each_allocation(lambda: xsum.xs_server_create(budget_bytes=1 << 30, streams=2))
    assert n == 5  # slots, then device and pinned batch buffers per stream
    try:
        rid = xsum.xs_server_submit(srv, d, d.numel())
        r = xsum.xs_server_wait(srv, rid, 60_000_000_000)
        assert f2b(r["value"]) == c_oracle.sum_bits(x)
    finally:
        xsum.xs_server_destroy(srv)


def test_serial_replay_session(data):
    x, d = data
    base = d.data_ptr()
    items = [(0, 1, base, 1000, 0), (0, 1, base + 8000, x.size - 1000, xsum.XS_REQ_FINISH)]
    s = stream_with_workspace(d)
    (vals, _), n = fail_each_allocation(lambda: xsum.xs_serial_replay(items, s))
    assert n == 1  # the session's accumulator
    assert f2b(vals[1]) == c_oracle.sum_bits(x)
