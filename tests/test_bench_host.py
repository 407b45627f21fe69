"""Host logic of bench.py (no GPU): workload names, the algorithmic-byte model, the gating of the
committed ncu records by kernel sources and launch settings, the bounded oracle sample, and the
reference arm (the CPU oracle) end to end."""

import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
import workloads as w  # noqa: E402


def test_workload_names():
    j = bench.get_workload("s11_lrx")
    assert (j.n, j.k, j.inverse_closed) == (11, 3, True)
    j = bench.get_workload("pancake:14")
    assert j.n == 14 and j.k == 13 and j.start is None and j.name == "S14-pancake-k13-full"
    j = bench.get_workload("lrx:32:bin")
    assert j.start == w.binary_start(32) and j.name.startswith("Bin32-lrx")
    with pytest.raises(ValueError):
        bench.get_workload("no-such-workload")


def test_algorithmic_bytes_and_neighbours():
    layers = [1, 3, 2]          # a complete growth with k = 2
    # B_r = 8 F_r + 16 k F_r + 8 (F_r + F_{r-1}) + 8 F_{r+1}, summed over the expanded layers
    want = (8 + 32 + 8 + 24) + (24 + 96 + 32 + 16) + (16 + 64 + 40 + 0)
    assert bench.algorithmic_bytes(layers, 2, True) == want
    assert bench.neighbours(layers, 2, True) == 2 * 6
    assert bench.neighbours(layers, 2, False) == 2 * 4            # the last layer not expanded
    # S_11 LRX: the 3.19 GB per growth quoted with the roofline
    g = [int(l.split()[1]) for l in open(os.path.join(ROOT, "tests", "golden", "s11_lrx_growth.txt"))
         if not l.startswith("#")]
    assert abs(bench.algorithmic_bytes(g, 3, True) / 1e9 - 3.193) < 0.001


def test_ncu_records_are_gated():
    import hashlib
    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name, rec in recs.items():
        h = hashlib.sha256()
        for src in rec["kernel_sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        current = h.hexdigest() == rec["kernel_sources_sha256"]
        got = bench.measured_record(name, rec["workload"], rec.get("settings"))
        assert (got is not None) == current          # a record is used only while its sources match
        if current:
            assert bench.measured_traffic(name, rec["workload"], rec.get("settings")) == rec["dram_bytes"]
        assert bench.measured_record(name, "another workload") is None
        if "settings" in rec:
            other = dict(rec["settings"], wave_l2=12345)
            assert bench.measured_record(name, rec["workload"], other) is None
    assert bench.measured_record("no_such_kernel<1>", "S11-LRX-k3-full") is None


def test_dram_rate_from_the_ncu_traffic():
    roof = bench.with_dram_rate({"traffic": 270_000_000, "kernel_ms": 1.5, "peak": 6750.0})
    assert abs(roof["traffic_gbs"] - 180.0) < 1e-9 and abs(roof["traffic_frac"] - 180.0 / 6750.0) < 1e-12
    assert "traffic_gbs" not in bench.with_dram_rate({"traffic": None, "kernel_ms": 1.5, "peak": 1.0})


def test_sample_radius_bounds_the_oracle():
    assert bench.sample_radius(bench.get_workload("s8_coxeter"), 10.0) == -1   # whole growth fits
    r = bench.sample_radius(bench.get_workload("pancake:12"), 1.0)
    assert 1 <= r < 14


def test_reference_arm_runs_the_oracle():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "s8_coxeter", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["steps"] == 2 and line["warmup"] == 3
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "batch"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode == 0 and "unavailable" in json.loads(out.stdout.strip().splitlines()[-1])


def test_generated_candidates_after_the_parent_edge_skip():
    import bench
    import workloads as w
    lay = [1, 3, 6, 12]
    # LRX: every generator's inverse is in the set, so each state after the first expands k - 1
    assert bench.generated_candidates(5, w.lrx(5), lay, True, True) == 3 + 2 * (3 + 6 + 12)
    assert bench.generated_candidates(5, w.lrx(5), lay, True, False) == 3 * sum(lay)
    assert bench.generated_candidates(5, w.lrx(5), lay, False, True) == 3 + 2 * (3 + 6)
    # LX is directed (L's inverse R is missing; X is an involution): it depends on the path
    assert bench.generated_candidates(5, w.lx(5), lay, True, True) is None
    # a directed set with no inverse present: nothing is skipped
    c = w.cycle(5, [0, 1, 2, 3, 4])
    assert bench.generated_candidates(5, [c], lay, True, True) == sum(lay)
    # n = 16 keys carry no tag
    assert bench.generated_candidates(16, w.coxeter(16), lay, True, True) == 15 * sum(lay)
