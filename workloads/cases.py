"""Runs one library entry point on one synthetic workload (for timing and ncu).

    python -m workloads.cases <case> [--reps N] [--prefetch TILES]

Cases: sum_cfg1 (the default method), small_cfg1 and large_cfg1 (each method
explicitly), sum_cfg2a (2^28 doubles, full exponent range) and small_cfg2a (the same
with the small method), mean_cfg1, dot_cfg1, norm2_cfg1, f32_2e8,
seg_cfg3_5k (5,000 segments of the config-3 length law), seg_cfg3 (all
100,000, 58 GB, default options), serve_cfg4 (300 one-shot
requests of the serving recipe, log-uniform 1e3..1e8 values from three value
recipes, through one server), seg_tiny (2,000,000
segments of 1..100 values). Inputs are generated on the device; the case prints
its median CUDA-event time. This module only calls the library.
"""

from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


CASES = ("sum_cfg1", "small_cfg1", "sum_cfg2a", "small_cfg2a", "mean_cfg1", "large_cfg1", "dot_cfg1", "norm2_cfg1", "dot_small_cfg1", "norm2_small_cfg1", "f32_2e8", "f32_small_2e8",
         "seg_cfg3_5k", "seg_cfg3", "seg_tiny", "serve_cfg4")


def build_case(name: str):
    if name not in CASES:
        raise SystemExit(f"unknown case {name}")
    import numpy as np
    import torch

    from paper_1505_05571_gb300 import xsum
    from workloads import devgen, gen

    dev = torch.device("cuda", 0)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    if name in ("sum_cfg2a", "small_cfg2a"):  # exponents uniform over the full range, subnormals included
        n = 1 << 28
        x = torch.empty(n, dtype=torch.int64, device=dev)
        devgen.full_range(x, 0, 0)
        m = xsum.XS_METHOD_AUTO if name == "sum_cfg2a" else xsum.XS_METHOD_SMALL
        return (lambda: xsum.xs_sum_async(x.view(torch.float64), n, out, m)), 8 * n, (x,)
    if name in ("sum_cfg1", "small_cfg1", "mean_cfg1", "large_cfg1", "dot_cfg1", "norm2_cfg1", "dot_small_cfg1",
                "norm2_small_cfg1"):
        n = 10 ** 8
        x = torch.empty(n, dtype=torch.int64, device=dev)
        devgen.band(x, 0, 0)
        xd = x.view(torch.float64)
        if name == "sum_cfg1":
            return (lambda: xsum.xs_sum_async(xd, n, out)), 8 * n, (x,)
        if name == "mean_cfg1":
            return (lambda: xsum.xs_mean_async(xd, n, out)), 8 * n, (x,)
        if name == "small_cfg1":
            return (lambda: xsum.xs_sum_async(xd, n, out, xsum.XS_METHOD_SMALL)), 8 * n, (x,)
        if name == "large_cfg1":
            return (lambda: xsum.xs_sum_async(xd, n, out, xsum.XS_METHOD_LARGE)), 8 * n, (x,)
        if name == "norm2_cfg1":
            return (lambda: xsum.xs_norm2_async(xd, n, out)), 8 * n, (x,)
        if name == "norm2_small_cfg1":
            return (lambda: xsum.xs_norm2_method_async(xd, n, out, xsum.XS_METHOD_SMALL)), 8 * n, (x,)
        y = torch.empty(n, dtype=torch.int64, device=dev)
        devgen.band(y, 1, 0)
        yd = y.view(torch.float64)
        if name == "dot_small_cfg1":
            return (lambda: xsum.xs_dot_method_async(xd, yd, n, out, xsum.XS_METHOD_SMALL)), 16 * n, (x, y)
        return (lambda: xsum.xs_dot_async(xd, yd, n, out)), 16 * n, (x, y)
    if name in ("f32_2e8", "f32_small_2e8"):
        m = 2 * 10 ** 8
        rng = np.random.default_rng(0)
        h = ((rng.integers(67, 187, m, dtype=np.uint32) << np.uint32(23))
             | rng.integers(0, 1 << 23, m, dtype=np.uint32)
             | (rng.integers(0, 2, m, dtype=np.uint32) << np.uint32(31)))
        f = torch.from_numpy(h.view(np.int32)).to(dev)
        o32 = torch.empty(1, dtype=torch.float32, device=dev)
        fd = f.view(torch.float32)
        if name == "f32_small_2e8":
            return (lambda: xsum.xs_sum_f32_method_async(fd, m, o32, xsum.XS_METHOD_SMALL)), 4 * m, (f,)
        return (lambda: xsum.xs_sum_f32_async(fd, m, o32)), 4 * m, (f,)
    if name in ("seg_cfg3_5k", "seg_cfg3", "seg_tiny"):
        if name == "seg_cfg3_5k":
            lengths = gen.cfg3_lengths(0, 5000, 10 ** 6)
        elif name == "seg_cfg3":
            lengths = gen.cfg3_lengths(0, 100_000, 10 ** 6)
        else:
            lengths = np.random.default_rng(0).integers(1, 101, 2_000_000).astype(np.int64)
        off = gen.cfg3_offsets(lengths)
        total = int(off[-1])
        v = torch.empty(total, dtype=torch.int64, device=dev)
        devgen.band(v, 0, 0, -30, 30)
        od = torch.from_numpy(off).to(dev)
        so = torch.empty(lengths.size, dtype=torch.float64, device=dev)
        plan = xsum.xs_seg_plan_create(v.view(torch.float64), od, lengths.size, so)
        return (lambda: xsum.xs_seg_plan_launch(plan)), 8 * total, (v, od, so)
    if name == "serve_cfg4":
        R = 1 << 27
        arena = torch.empty(3 * R, dtype=torch.int64, device=dev)
        devgen.band(arena[:R], 3, 0, -40, 40)
        devgen.band(arena[R:2 * R], 4, 0, -60, 60)
        devgen.paired(arena[2 * R:], 5, 0)
        rng = np.random.default_rng(7)
        items, total = [], 0
        for _ in range(300):
            nn = int(np.exp(rng.uniform(np.log(1e3), np.log(1e8))))
            o = int(rng.integers(0, R - nn)) + int(rng.integers(0, 3)) * R
            items.append((0, 0, arena.data_ptr() + 8 * o, nn, 0))
            total += nn
        # one batch may take every request that is pending when it is formed
        srv = xsum.xs_server_create(budget_bytes=40 << 30, streams=3, max_batch=1024)

        def run():
            ids, _ = xsum.xs_server_replay(srv, items)
            for i in ids:
                xsum.xs_server_wait(srv, i, 120_000_000_000)
        return run, 8 * total, (arena,)
    raise SystemExit(f"unknown case {name}")


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=CASES)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--prefetch", type=int, default=None,
                    help="L2 prefetch distance in tiles (library default if absent)")
    args = ap.parse_args()
    if args.prefetch is not None:
        from paper_1505_05571_gb300 import xsum

        xsum.xs_set_prefetch_tiles(args.prefetch)
    fn, nbytes, _keep = build_case(args.case)
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    t = times[len(times) // 2]
    pf = "" if args.prefetch is None else f" (prefetch {args.prefetch})"
    print(f"{args.case}{pf}: {t * 1000:.1f} us, {nbytes / (t * 1e-3) / 1e9:.1f} GB/s")


if __name__ == "__main__":
    main()
