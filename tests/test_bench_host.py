"""Host-side pieces of bench.py that need no GPU: the measured peak, the
kernel hash that ties the committed ncu summary to the kernel sources, and
the traffic lookup that must go null when they no longer match."""
import json
import re

import pytest

import bench


def test_measured_peak_is_the_driver_written_copy_bandwidth():
    peak, source = bench.measured_peak()
    with open(bench.PEAKS_FILE) as fh:
        assert peak == pytest.approx(float(json.load(fh)["hbm_gbs"]))
    assert source == "measured"


def test_kernel_sha_covers_the_headline_kernel_sources():
    sha = bench.kernel_sha()
    assert re.fullmatch(r"[0-9a-f]{16}", sha)
    assert any(p.endswith("rd_step_kernel.cuh") for p in bench.KERNEL_SOURCES)


def _profile_sha():
    text = open(bench.PROFILE_FILE).read()
    return re.search(r"kernel_sha: `([0-9a-f]{16})`", text).group(1)


def test_traffic_is_reported_only_for_the_profiled_kernel_and_tile(monkeypatch):
    monkeypatch.setattr(bench, "kernel_sha", _profile_sha)
    text = open(bench.PROFILE_FILE).read()
    tile_y = int(re.search(r"- tile_y: (\d+)", text).group(1))
    dram = float(re.search(r"- dram_bytes_per_launch: (\d+)", text).group(1))
    traffic, tun = bench.profiled_traffic(1, 16, tile_y)
    assert traffic == dram and tun["tile_y"] == tile_y
    # another tile height, or kernel sources changed since the capture: null
    assert bench.profiled_traffic(1, 16, tile_y + 2) == (None, None)
    monkeypatch.setattr(bench, "kernel_sha", lambda: "0" * 16)
    assert bench.profiled_traffic(1, 16, tile_y) == (None, None)


def test_whole_job_rate_and_roofline_entry():
    assert bench.whole_job_glups(3e9, 4, 2.0) == pytest.approx(6.0)
    peak, _ = bench.measured_peak()
    e = bench._entry(cells=1_000_000, steps=1000, seconds=0.5, bytes_per_cell_step=16)
    assert e["glups"] == pytest.approx(2.0)
    assert e["roofline_frac"] == pytest.approx(2.0 * 16 / peak)
