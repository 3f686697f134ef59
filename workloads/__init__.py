"""Seeded synthetic inputs for exact FP64 summation.

This package generates the arrays that both the CPU oracle tests and the CUDA
path consume. It holds none of the summation method's arithmetic: it only turns
counter-based random bits into IEEE-754 binary64 bit patterns, segment lengths
and request schedules.

Every value is a pure function of (seed, stream, index) through SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), so any index range of any workload can be regenerated on its own,
on the host here or on the device by the CUDA twin in ``workloads/csrc``.
"""

from .gen import (  # noqa: F401
    GAMMA,
    MASK64,
    mix64_int,
    stream_key,
    draws,
    bits_to_f64,
    f64_to_bits,
    pow2_band_bits,
    full_range_bits,
    cfg0_cancel,
    cfg1_band,
    cfg2a_full_range,
    cfg2a_paired,
    cfg2b_cancel_1e300,
    cfg2c_repeat,
    cfg2d_side_cases,
    cfg3_lengths,
    cfg3_offsets,
    cfg3_values,
    zero_sum_mirror,
    affine_perm_inverse,
    STREAMS,
)
