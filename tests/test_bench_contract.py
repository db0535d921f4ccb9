"""The benchmark's host side on the CPU: the reference arm's JSON line (the oracle timed on the
host cores) and the work figures the GPU arm's rooflines are built from."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--ref-L", "32"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["value"] > 0 and line["ms_per_step"] > 0
    # the config names the lattice actually run, a bounded sample of the GPU arm's workload
    assert line["config"]["L"] == 32 and line["config"]["N"] == 32 * 32
    assert line["config"]["workload"].startswith("L=32 ")
    assert line["config"]["sample_of"] == {"L": 2304, "N": 2304 * 2304}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "L=32" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_block_local_levels():
    # KW levels 1..p0 run block-locally while a level-p0 group (g 2^p0 vertices) fits 4096
    # and the palette fits 64 colours; at L = 2304, T = 0.6D the graph has Delta = 38 (g = 39)
    # and M = ceil(log2 ceil(N / g)) = 18 levels, of which the library reports 6 block-local
    assert bench.low_levels(39, 18) == 6
    assert bench.low_levels(64, 20) == 6
    assert bench.low_levels(65, 20) == 0   # palette above 64: no block-local levels
    assert bench.low_levels(4096, 3) == 0  # a level-1 group would exceed 4096
    assert bench.low_levels(3, 2) == 2     # capped by the number of levels


def test_algorithmic_work_figures():
    k, M, p0 = 17.8, 18, 6
    b = bench.algorithmic_bytes(k, M, p0)
    assert abs(b["switch"] - (40 + 16 * k)) < 1e-9
    assert abs(b["colour"] - ((4 + 4 * k + 9) + (M - p0) * (4 + 2 * k) + 12)) < 1e-9
    assert abs(b["sweep"] - (60 + 8 * k)) < 1e-9
    # the FP64 form's pair cache: 16-byte records and 4-byte ids written by switch and fill,
    # read (and half written) by the sweep
    c = bench.algorithmic_bytes(k, M, p0, cache=True)
    assert abs(c["switch"] - (40 + 28 * k)) < 1e-9 and abs(c["sweep"] - (60 + 36 * k)) < 1e-9
    assert c["colour"] == b["colour"]
    # no block-local level: every level reads half the rows
    assert abs(bench.algorithmic_bytes(k, M, 0)["colour"] - (M * (4 + 2 * k) + 12)) < 1e-9
    f = bench.algorithmic_flops(k, 14.4)
    assert f["colour"] == 0.0
    # the sweep's plan per pair endpoint: two pair energies and one pseudointeraction term (the
    # other is read from the pair cache)
    assert abs(f["switch"] - 51 * 14.4) < 1e-9 and abs(f["sweep"] - 70 * k) < 1e-9


def test_cooling_schedule_and_cell_splits():
    # Sec. 3.1: from 1.25 J down to 0.05 J in steps of 0.05 J (25 temperatures)
    s = bench.cooling_schedule()
    assert len(s) == 25 and s[0] == 1.25 and s[-1] == 0.05
    assert all(abs((a - b) - 0.05) < 1e-9 for a, b in zip(s, s[1:]))
    assert set(bench.TABLE1) <= set(s)
    for nproc, (cx, cy) in bench.CELL_SPLITS.items():
        assert cx * cy == nproc and cx <= cy
