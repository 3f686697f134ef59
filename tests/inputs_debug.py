"""Inputs of the checked-build test (bit patterns), shared by the test and the
child process it starts: arrays that drive every path of the single-array
kernels near their bounds, and a mixed-length segmented workload."""

import numpy as np

import workloads as W


def cases() -> dict:
    out = {"cfg0": W.f64_to_bits(W.cfg0_cancel(0))}
    # same-sign terms at the top of a chunk (e & 31 == 31) with zeros and
    # subnormals every 61 values: carries reach their bound between propagations
    n = 3_000_017
    rng = np.random.default_rng(61)
    x = (np.uint64(0x7DF) << np.uint64(52)) | rng.integers(0, 1 << 52, n, dtype=np.uint64)
    rare = np.array([0, 0x8000000000000000, 1, 0x800FFFFFFFFFFFFF, 0x0008000000000000], dtype=np.uint64)
    sel = np.arange(30, n, 61)
    x[sel] = rare[rng.integers(0, rare.size, sel.size)]
    out["top_of_chunk_rare"] = x
    out["repeat_0.1"] = np.full(1_000_003, W.f64_to_bits(np.array([0.1]))[0], dtype=np.uint64)
    out["full_range"] = W.cfg2a_full_range(3, 0, 1 << 22)
    out["band_2^25+3"] = W.cfg1_band(4, 0, (1 << 25) + 3)
    sub = rng.integers(0, 1 << 52, 100_001, dtype=np.uint64)
    sub |= rng.integers(0, 2, sub.size, dtype=np.uint64) << np.uint64(63)
    out["subnormals"] = sub
    spec = W.cfg1_band(5, 0, 200_000)
    spec[1234] = 0x7FF0000000000000
    spec[99_999] = 0xFFF8000000000abc
    out["inf_nan"] = spec
    return out


def segmented():
    rng = np.random.default_rng(9)
    lengths = W.cfg3_lengths(9, 700, 200_000)
    special = np.array([0, 1, 2, 3, 31, 32, 33, 64, 65, 4096, 4097, 8191, 8193, 12289], dtype=np.int64)
    lengths[rng.integers(0, lengths.size, special.size)] = special
    off = W.cfg3_offsets(lengths)
    return W.cfg3_values(9, 0, int(off[-1])), off
