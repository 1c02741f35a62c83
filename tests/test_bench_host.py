"""Host logic of bench.py (no GPU): the instruction-issue bound, the rule that a figure from a
committed ncu summary is used only when it was taken on the current kernel sources, and the
reference arm's split of its K steps over the host's processes."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_issue_bound_arithmetic():
    assert bench.issue_bound(1000.0, None) is None
    b = bench.issue_bound(40000.0, 1.5e6)
    peak = 152 * 4 * 2.07e9
    assert b["frac"] == pytest.approx(40000.0 * 1.5e6 / peak, rel=1e-12)
    assert b["max_frames_per_s"] == pytest.approx(peak / 1.5e6, rel=1e-12)
    assert b["achieved"] == pytest.approx(6.0e10 / 1e12, rel=1e-12)


def test_profile_figures_are_used_only_on_their_kernel_sources(tmp_path):
    sha = bench.kernel_source_sha()
    good = tmp_path / "good.md"
    good.write_text(f"warp_inst_per_launch: 1234567\nkernel_source_sha: {sha}\n")
    assert bench.profiled_value("warp_inst_per_launch", str(good)) == 1234567.0
    assert bench.profiled_value("dram_bytes_per_launch", str(good)) is None  # key absent
    stale = tmp_path / "stale.md"
    stale.write_text("warp_inst_per_launch: 1234567\nkernel_source_sha: 0000000000000000\n")
    assert bench.profiled_value("warp_inst_per_launch", str(stale)) is None
    assert bench.profiled_value("warp_inst_per_launch", str(tmp_path / "missing.md")) is None
    # the staged summary is keyed on its own sources
    assert bench.kernel_source_sha(bench.KERNEL_SOURCES_STAGED) != sha


@pytest.mark.parametrize("k,cores,cap", [(1, 16, 100), (2, 16, 100), (20, 16, 100), (1000, 16, 100),
                                         (33, 8, 100), (7, 1, 3)])
def test_reference_arm_spreads_exactly_k_frames(k, cores, cap):
    counts = bench.reference_counts(k, cores, cap)
    assert 1 <= len(counts) <= min(cores, k)
    assert all(1 <= c <= cap for c in counts)
    assert max(counts) - min(counts) <= 1 or max(counts) == cap
    if k <= cap * len(counts):
        assert sum(counts) == k  # exactly the K requested frames unless the cap bounds them
    else:
        assert all(c == cap for c in counts)
