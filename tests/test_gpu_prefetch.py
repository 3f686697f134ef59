"""The L2 prefetch distance is a pure scheduling choice: every kernel family
that takes it returns the oracle's bits at every distance."""

import pytest

import workloads as W
from oracle import c_oracle, products
from paper_1505_05571_gb300 import xsum
from tests.gpu_util import bits_of, out_slot, to_device
from tests.test_gpu_f32 import gpu32
from tests.test_oracle32 import rand32

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def restore_default():
    yield
    xsum.xs_set_prefetch_tiles(-1)


@pytest.mark.parametrize("tiles", [0, 1, 3, 8, 64])
def test_all_families_at_every_distance(tiles):
    n = 2_000_003
    x = W.gen.cfg1_band(7, 0, n)
    y = W.gen.cfg1_band(8, 0, n)
    xsum.xs_set_prefetch_tiles(tiles)
    dx, dy = to_device(x, 1), to_device(y, 0)
    out = out_slot()
    xsum.xs_sum_async(dx, n, out)
    assert int(bits_of(out)[0]) == c_oracle.sum_bits(x)
    xsum.xs_dot_async(dx, dy, n, out)
    assert int(bits_of(out)[0]) == products.dot_bits(x, y)
    xsum.xs_norm2_async(dy, n, out)
    assert int(bits_of(out)[0]) == products.norm2_bits(y)
    f = rand32(9, 3 * n + 1)
    assert gpu32(f, 2) == c_oracle.sum_f32_bits(f)
