"""The committed ncu summaries: their commands run committed files only, and the
per-launch DRAM figures are tied to the kernel code they were taken on."""

import glob
import json
import os
import re
import subprocess
import sys

import bench
from workloads import cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
CSRC = os.path.join(ROOT, "paper_1505_05571_gb300", "csrc")


def _text(p):
    with open(p) as fh:
        return fh.read()


def test_profile_commands_name_existing_cases_kernels_and_flags():
    assert PROFILES
    kernels = "".join(_text(p) for p in glob.glob(os.path.join(CSRC, "*.cu*")))
    bench_help = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                                capture_output=True, text=True, check=True).stdout
    for p in PROFILES:
        t = _text(p)
        for name in re.findall(r"python -m workloads\.cases (\w+)", t):
            assert name in cases.CASES, (p, name)
        for k in re.findall(r"-k regex:(\w+)", t):
            assert re.search(r"__global__[^;{]*\b%s\s*\(" % k, kernels), (p, k)
        for line in re.findall(r"python bench\.py([^\n`]*)", t):
            for flag in re.findall(r"--[\w-]+", line):
                assert flag in bench_help, (p, flag)


def test_traffic_entries_point_at_summaries_of_known_kernels():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    assert "k_sum_small" in d
    for k, e in d.items():
        assert k in bench.KERNEL_SOURCES
        assert os.path.exists(os.path.join(ROOT, "profiles", e["capture"]))
        assert e["dram_bytes_per_launch"] == e["dram_read_bytes"] + e["dram_write_bytes"]
        assert len(e["source_hash"]) == 16


def test_code_hash_ignores_comments_only():
    a = "int f(int x) {  // doubles\n  return 2 * x;\n}\n"
    b = "// a new header comment\nint f(int x) {\n\n  return 2 * x;  // same code\n}\n"
    c = "int f(int x) {\n  return 3 * x;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_stale_profile_gives_no_traffic(monkeypatch):
    k = "k_sum_small"
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        committed = json.load(fh)[k]["dram_bytes_per_launch"]
    assert bench.profiled_traffic(k) in (None, committed)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "0" * 16)
    assert bench.profiled_traffic(k) is None
