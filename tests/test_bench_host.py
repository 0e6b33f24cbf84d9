"""Host-side pieces of bench.py: the committed ncu summary it reads the
headline kernel's DRAM traffic from, and the source-hash gate on it."""
import os
import re

import bench


def _recorded(key):
    path = os.path.join(bench.ROOT, "profiles", "fwd_sweep_f64_2048x2048x64.md")
    with open(path) as f:
        m = re.search(rf"- {key}: `([^`]+)`", f.read())
    assert m, f"{key} missing from the headline summary"
    return m.group(1)


def test_headline_summary_records_traffic_and_hash():
    traffic = float(_recorded("dram_bytes_per_launch"))
    algorithmic = 48 * bench.SHAPE[0] * bench.SHAPE[1] * bench.SHAPE[2]
    # the sweep reads and writes each field once: DRAM bytes within a few % of 48 B/point
    assert 0.95 * algorithmic <= traffic <= 1.05 * algorithmic
    assert re.fullmatch(r"[0-9a-f]{16}", _recorded("source_sha1"))


def test_traffic_is_used_only_for_the_recorded_source():
    h = _recorded("source_sha1")
    assert bench.profile_traffic("fwd_sweep", h) == float(_recorded("dram_bytes_per_launch"))
    assert bench.profile_traffic("fwd_sweep", "0" * 16) is None
    assert bench.profile_traffic("no_such_kernel", h) is None


def test_kernel_source_hash_covers_existing_files():
    csrc = os.path.join(bench.ROOT, "paper_2010_01545_gb300", "csrc")
    for name in bench.FWD_KERNEL_SOURCES:
        assert os.path.exists(os.path.join(csrc, name)), name
    assert re.fullmatch(r"[0-9a-f]{16}", bench.kernel_source_hash())


def test_all_cores_oracle_leg_reports_threads_and_rate():
    import workload
    grid = workload.vertical_grid(bench.SHAPE[2])
    planes = 6
    winds = [workload.wind_field(planes + 2, bench.SHAPE[1], bench.SHAPE[2], f) for f in range(3)]
    leg = bench.oracle_all_cores(winds, grid, planes)
    if "unavailable" in leg:
        return
    assert leg["cores"] >= 1 and leg["value"] > 0 and leg["unit"] == bench.UNIT
    assert f"{planes} x-planes" in leg["sample"]
