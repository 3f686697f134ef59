"""The checked build (-DXS_DEBUG): on the same inputs as the parity tests, every
kernel path gives the oracle's bits and no check fails.

The debug library is built on demand (build.build(debug=True)) and loaded in a
fresh process, so it never mixes with the release library of this one. The
child prints the bit patterns it got; the oracle is computed here.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import c_oracle, products
from paper_1505_05571_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
from paper_1505_05571_gb300 import build, xsum
xsum.load(build.LIB_DEBUG)
from tests.inputs_debug import cases, segmented
assert xsum.xs_is_debug_build()
out = torch.empty(1, dtype=torch.float64, device="cuda")
res = {}
for name, bits in cases().items():
    d = torch.from_numpy(bits.view(np.int64)).cuda().view(torch.float64)
    for m in (xsum.XS_METHOD_AUTO, xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE):
        xsum.xs_sum_async(d, d.numel(), out, m)
        res[f"{name}/{m}"] = int(out.view(torch.int64).item()) & ((1 << 64) - 1)
    if d.numel() <= 1 << 22:  # products: x against x reversed, both methods
        dr = d.flip(0).contiguous()
        for m in (xsum.XS_METHOD_SMALL, xsum.XS_METHOD_LARGE):
            xsum.xs_dot_method_async(d, dr, d.numel(), out, m)
            res[f"{name}/dot/{m}"] = int(out.view(torch.int64).item()) & ((1 << 64) - 1)
vals, off = segmented()
vd = torch.from_numpy(vals.view(np.int64)).cuda().view(torch.float64)
od = torch.from_numpy(off).cuda()
so = torch.empty(off.size - 1, dtype=torch.float64, device="cuda")
for k, opts in enumerate((None, {"block": 128, "unroll": 8, "tile_elems": 4096, "short_max": 64},
                          {"block": 32, "unroll": 8, "tile_elems": 1 << 20, "short_max": 0})):
    p = xsum.xs_seg_plan_create(vd, od, off.size - 1, so, opts)
    xsum.xs_seg_plan_launch(p)
    torch.cuda.synchronize()
    xsum.xs_seg_plan_destroy(p)
    res[f"seg/{k}"] = [int(b) for b in so.view(torch.int64).cpu().numpy().view(np.uint64)]
res["status"] = xsum.xs_debug_status()
print(json.dumps(res))
"""


def test_debug_build_matches_oracle_and_no_check_fails():
    build.build(debug=True)
    from tests.inputs_debug import cases, segmented

    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert got.pop("status") == 0
    for name, bits in cases().items():
        expect = c_oracle.sum_bits(bits)
        for m in (0, 1, 2):
            assert got[f"{name}/{m}"] == expect, (name, m)
        if bits.size <= 1 << 22:
            expect_dot = products.dot_bits(bits, bits[::-1].copy())
            for m in (1, 2):
                assert got[f"{name}/dot/{m}"] == expect_dot, (name, "dot", m)
    vals, off = segmented()
    expect = [int(b) for b in c_oracle.segment_sums_bits(vals, off)]
    for k in range(3):
        assert got[f"seg/{k}"] == expect, k
