"""Host arithmetic of bench.py's roofline entry: the committed ncu traffic
of the plasma pass scaled to a workload, and the issue and L1 fractions
derived from its per-row counts (no GPU)."""
import json
import os

import pytest

import bench


def committed():
    return json.load(open(os.path.join(bench.ROOT, "profiles", "k_dpd_traffic.json")))


def test_traffic_is_the_channel_capture_scaled_by_rows_for_the_paper_system():
    d = committed()
    if d["channel"]["source_hash"] != bench.kernel_source_hash():
        pytest.skip("the committed capture predates the kernel source")
    n = 101003469
    b, note = bench.traffic_entry("paper", d["channel"]["skin"], n)
    assert b == pytest.approx(d["channel"]["dram_bytes_per_launch"] * n / d["channel"]["rows"])
    assert "scaled" in note
    b, note = bench.traffic_entry("channel", d["channel"]["skin"], d["channel"]["rows"])
    assert b == pytest.approx(d["channel"]["dram_bytes_per_launch"])
    assert bench.traffic_entry("channel", d["channel"]["skin"] + 0.1, 1)[0] is None   # another skin: no figure


def test_limiter_fractions_follow_the_per_row_counts():
    d = committed()
    if d["instructions"]["source_hash"] != bench.kernel_source_hash():
        pytest.skip("the committed capture predates the kernel source")
    n, ms, mhz = 1_000_000, 0.1, 2000.0
    lim = bench.issue_limiter("channel", ms, n, mhz)
    per_row = d["instructions"]["warp_inst_per_row"]
    assert lim["issue_fraction"] == pytest.approx(per_row * n / (ms * 1e-3) / (152 * 4 * mhz * 1e6))
    wf = d["channel"]["l1_wavefronts_per_launch"] / d["channel"]["rows"]
    assert lim["l1_wavefront_fraction"] == pytest.approx(wf * n / (ms * 1e-3) / (152 * mhz * 1e6))
    assert bench.issue_limiter("channel", ms, n, None) is None     # no clock sample, no fraction
