"""Host-side pieces of bench.py that need no GPU: the measured peak, the
kernel hash that ties the committed ncu summary to the kernel sources, the
traffic lookup that must go null when they no longer match, the summary of
the clock samples (median SM clock under load, throttle reasons) and the
tuning argument."""
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


def _sampler_with(rows):
    s = bench.ClockSampler(0)
    s.tmp.write("".join(r + "\n" for r in rows))
    return s


def test_clock_summary_takes_the_median_under_load_and_every_reason():
    # nvidia-smi rows: index, sm, max sm, power, active mask, hw slowdown,
    # hw thermal, sw thermal, sw power cap
    rows = [
        "0, 345, 2070, 180.5, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1399.9, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 10, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "garbage line",                                                            # skipped
    ]
    out = _sampler_with(rows).summary()
    # the idle sample (below half the maximum) is left out of the median
    assert out["sm_mhz"] == 2055
    assert out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 4


def test_clock_summary_names_the_throttle_reasons_that_reject_a_run():
    rows = [
        "0, 1500, 2070, 1200, 0x8, Active, Not Active, Not Active, Not Active",
        "0, 1600, 2070, 1200, 0x40, Not Active, Active, Not Active, Not Active",
        "0, 1700, 2070, 1200, 0x20, Not Active, Not Active, Active, Not Active",
    ]
    out = _sampler_with(rows).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1600


def test_clock_summary_without_samples_says_so():
    out = _sampler_with([]).summary()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_tuning_argument():
    assert bench.parse_tuning("1,14,64") == dict(tsteps=1, tile_y=14, zchunk=64, regcap=0)
    assert bench.parse_tuning("2,8,32,1,8") == dict(tsteps=2, tile_y=8, zchunk=32, regcap=1,
                                                    tile_q=8)
    with pytest.raises(ValueError):
        bench.parse_tuning("1,x,64")


def test_every_profile_command_names_a_bench_workload_and_a_valid_tuning():
    import glob
    import os
    files = sorted(glob.glob(os.path.join(os.path.dirname(bench.PROFILE_FILE), "*.md")))
    assert files
    for path in files:
        text = open(path).read()
        # the command block: the lines after "Command" up to the first blank line
        cmd = " ".join(text.split("Command", 1)[1].split("\n\n")[1].replace("\\", " ").split())
        assert "--clock-control none" in cmd, path
        assert "python bench.py" in cmd, path
        src = open(bench.__file__).read()
        for flag in re.findall(r"(--[a-z][a-z-]*)", cmd.split("python bench.py", 1)[1]):
            assert f'add_argument("{flag}"' in src, (path, flag)
        m = re.search(r"--profile-workload (\S+)", cmd)
        if m:
            assert m.group(1) in bench.PROFILE_WORKLOADS, path
        m = re.search(r"--tuning (\S+)", cmd)
        if m:
            bench.parse_tuning(m.group(1))
