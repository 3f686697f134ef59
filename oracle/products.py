"""Oracle of the exact dot product and squared norm (test infrastructure only).

The paper computes each product with an ordinary floating-point multiply,
rounded to the nearest double, and sums the products exactly (performance
section, squared norm and dot product). Here the products come from numpy's
IEEE float64 multiply (a library primitive, pinned in the tests against Python's
own float multiply); a NaN product counts as the default quiet NaN
0x7FF8000000000000 (reading: NaN payloads of a multiply are processor-defined).
The sum of the products is the exact-sum oracle of this package.
"""

from __future__ import annotations

import numpy as np

from . import c_oracle

DEFAULT_NAN = 0x7FF8000000000000


def product_bits(x_bits, y_bits) -> np.ndarray:
    x = np.ascontiguousarray(x_bits, dtype=np.uint64).view(np.float64)
    y = np.ascontiguousarray(y_bits, dtype=np.uint64).view(np.float64)
    with np.errstate(all="ignore"):
        p = x * y
    pb = p.view(np.uint64).copy()
    pb[np.isnan(p)] = np.uint64(DEFAULT_NAN)
    return pb


def dot_bits(x_bits, y_bits) -> int:
    return c_oracle.sum_bits(product_bits(x_bits, y_bits))


def norm2_bits(x_bits) -> int:
    return c_oracle.sum_bits(product_bits(x_bits, x_bits))
