"""Device-resident accumulator handles: append, merge, round, export/import.

Partial exact sums added chunkwise give the exact sum of the union (Discussion:
split, sum parts exactly, add the superaccumulators, round once).
"""

import numpy as np
import pytest

import workloads as W
from oracle import c_oracle
from oracle import xsum_oracle as xo
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, out_slot, to_device

pytestmark = pytest.mark.gpu


def rounded(h):
    out = out_slot()
    xsum.xs_acc_round(h, out)
    return int(bits_of(out)[0])


def test_empty_accumulator_is_plus_zero():
    h = xsum.xs_acc_create()
    assert rounded(h) == 0
    xsum.xs_acc_destroy(h)


def test_append_in_pieces_equals_one_shot():
    x = W.cfg2a_paired(7, 0, 2_000_003)
    expect = c_oracle.sum_bits(x)
    d = to_device(x)
    rng = np.random.default_rng(1)
    for trial in range(3):
        cuts = np.sort(rng.integers(0, x.size, size=rng.integers(1, 12)))
        edges = [0, *cuts.tolist(), x.size]
        h = xsum.xs_acc_create()
        for a, b in zip(edges[:-1], edges[1:]):
            xsum.xs_acc_add(h, d[a:b], b - a)
        assert rounded(h) == expect
        assert rounded(h) == expect  # rounding leaves the state unchanged
        xsum.xs_acc_destroy(h)


def test_merge_equals_concatenation():
    a = W.cfg2b_cancel_1e300(3, 0, 1_000_000)
    b = W.cfg1_band(3, 0, 777_777)
    da, db = to_device(a), to_device(b)
    ha, hb = xsum.xs_acc_create(), xsum.xs_acc_create()
    xsum.xs_acc_add(ha, da, da.numel())
    xsum.xs_acc_add(hb, db, db.numel())
    xsum.xs_acc_merge(ha, hb)
    assert rounded(ha) == c_oracle.sum_bits(np.concatenate([a, b]))
    assert rounded(hb) == c_oracle.sum_bits(b)  # src unchanged
    xsum.xs_acc_destroy(ha)
    xsum.xs_acc_destroy(hb)


def test_export_is_canonical_and_roundtrips():
    x = W.cfg2a_paired(9, 0, 300_001)
    d = to_device(x)
    h = xsum.xs_acc_create()
    xsum.xs_acc_add(h, d, d.numel())
    state = xsum.xs_acc_export(h)
    chunks = xsum.acc_state_chunks(state)
    st = xo.state_of_bits(x.tolist())
    assert chunks == xo.canonical_chunks(st)  # the oracle's unique normalised form
    h2 = xsum.xs_acc_create()
    xsum.xs_acc_import(h2, state)
    assert rounded(h2) == rounded(h) == xo.finish(st)
    xsum.xs_acc_destroy(h)
    xsum.xs_acc_destroy(h2)


def test_specials_and_signed_zero_through_handles():
    h = xsum.xs_acc_create()
    nz = to_device(np.full(10, 0x8000000000000000, dtype=np.uint64))
    xsum.xs_acc_add(h, nz, 10)
    assert rounded(h) == 0x8000000000000000
    xsum.xs_acc_add(h, to_device(np.array([0x7FF8000000000042], dtype=np.uint64)), 1)
    xsum.xs_acc_add(h, to_device(np.array([0x7FF0000000000000], dtype=np.uint64)), 1)
    assert rounded(h) == 0x7FF8000000000042
    xsum.xs_acc_init(h)
    assert rounded(h) == 0
    xsum.xs_acc_destroy(h)


def test_import_rejects_non_canonical():
    h = xsum.xs_acc_create()
    bad = bytearray(xsum.xs_acc_export(h))
    bad[0:8] = (1 << 40).to_bytes(8, "little")
    with pytest.raises(xsum.XsError):
        xsum.xs_acc_import(h, bytes(bad))
    xsum.xs_acc_destroy(h)
