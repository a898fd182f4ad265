"""Host logic of bench.py on the CPU: the clock record that decides whether a
run saw throttling, and the source hash that ties the recorded DRAM traffic to
the device code it was measured on."""
import json
import os

import bench

LINE = "0, {sm}, 2070, {w}, 0x0000000000000000, Not Active, Not Active, Not Active, {cap}"


def test_clock_summary_median_min_and_reasons():
    lines = [LINE.format(sm=2070, w=380.5, cap="Not Active"),
             LINE.format(sm=2070, w=390.0, cap="Not Active"),
             LINE.format(sm=1965, w=1400.0, cap="Active"),
             "garbage", ""]
    s = bench.ClockSampler.summarize(lines)
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070 and s["sm_min_mhz"] == 1965 and s["sm_max_mhz"] == 2070
    assert s["power_w"] == 390.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown():
    line = "0, 1500, 2070, 900, 0x0, Active, Active, Not Active, Not Active"
    s = bench.ClockSampler.summarize([line])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_summary_without_samples_is_none():
    assert bench.ClockSampler.summarize([]) is None
    assert bench.ClockSampler.summarize(["[N/A], [N/A]"]) is None


def test_source_hash_covers_the_device_code_only():
    names = sorted(os.path.basename(p) for p in bench.KERNEL_SOURCES)
    assert names == ["lbm_batch_kernels.cuh", "lbm_device.cuh", "lbm_kernels.cu"]
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    rec = json.load(open(bench.PROFILE_TRAFFIC))
    assert set(rec["storage"]) >= {"f32", "f16d"}
    for e in rec["storage"].values():
        assert e["dram_bytes_per_step"] == (e["dram_read_bytes_per_step"]
                                            + e["dram_write_bytes_per_step"])
        # DRAM traffic of one step is within 5 % of the algorithmic bytes.
        assert abs(e["dram_bytes_per_step"] / e["algorithmic_bytes_per_step"] - 1) < 0.05
