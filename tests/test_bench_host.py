"""Host logic of bench.py (CPU only): the evidence it attaches to its JSON
line from the committed profile summaries, and the FLOP counts it divides by."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_every_profile_summary_carries_its_counters():
    """Every profiles/*.md ends with machine-readable ncu counters naming its
    kernel, workload and duration; bench.ncu_profiles() parses them all, with
    numbers as numbers."""
    import bench
    got = bench.ncu_profiles()
    files = sorted(f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".md"))
    assert sorted(got) == files
    for name, kv in got.items():
        assert isinstance(kv.get("kernel"), str) and kv["kernel"], name
        assert isinstance(kv.get("workload"), str) and kv["workload"], name
        assert isinstance(kv.get("gpu__time_duration_ms"), float) and kv["gpu__time_duration_ms"] > 0, name
        for k, v in kv.items():
            if k.endswith("_sum") or k.startswith("launch__"):
                assert isinstance(v, int) and v >= 0, (name, k, v)


def test_traffic_is_taken_only_for_matching_sources():
    """roofline.traffic comes from the headline kernel's capture only while the
    hash of its sources equals the one recorded with the capture; then it is
    the recorded per-launch figure (scaled from the depth-4 capture)."""
    import bench
    path = os.path.join(ROOT, "profiles", "m2l_lists_fp64_p10_octree_l5.md")
    rec = {}
    for line in open(path):
        if ":" in line and line.split(":")[0].strip() in ("kernel_sources_sha256_16", "dram_bytes_per_launch"):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    assert set(rec) == {"kernel_sources_sha256_16", "dram_bytes_per_launch"}
    t = bench.ncu_traffic()
    if rec["kernel_sources_sha256_16"] == bench.kernel_hash():
        assert t == float(rec["dram_bytes_per_launch"])
    else:
        assert t is None


@pytest.mark.parametrize("p,flop", [(1, 2 * 1 * 2 * 3 + 14 * 2), (10, 6160)])
def test_m2l_flop_count(p, flop):
    """The algorithmic FLOP of one M2L of order p: 2p(p+1)(2p+1) for the swaps
    and the z-axis translation plus 14p(p+1) for scaling and rotations (6,160
    at p = 10, the figure the roofline fraction divides by)."""
    import bench
    assert bench.m2l_flop(p) == flop
