"""Host logic of bench.py that shapes the reported line, on CPU: the clock
and throttle-reason summary of the nvidia-smi samples, the staleness rule of
the committed DRAM traffic, the percentile used for p50/p99 and the derived
ALU peaks."""
import pytest

import bench


class _DoneProc:
    """Stands in for a finished nvidia-smi process."""
    stdout = iter(())

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _DoneProc()
    s.lines = list(lines)
    return s


def test_clock_summary_median_max_and_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler(lines).stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_hardware_slowdown():
    lines = ["0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active"] * 3
    out = _sampler(lines).stop()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_nvidia_smi():
    s = bench.ClockSampler(0)
    out = s.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_profile_traffic_is_dropped_once_the_sources_change(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "factor_fp64_w.txt").write_text("header line: with a colon\nsource_hash: abc123\n"
                                            "traffic_bytes_per_factor: 2.5e7\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "abc123")
    assert bench._profile_traffic("w", "fp64") == 2.5e7
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "other")
    assert bench._profile_traffic("w", "fp64") is None
    assert bench._profile_traffic("missing", "fp64") is None


def test_kernel_source_hash_covers_every_cuda_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2609_29977_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("x")
    (csrc / "b.cuh").write_text("y")
    (csrc / "notes.txt").write_text("z")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_source_hash()
    (csrc / "notes.txt").write_text("changed")
    assert bench._kernel_source_hash() == h0          # not a CUDA source
    (csrc / "b.cuh").write_text("y2")
    assert bench._kernel_source_hash() != h0          # a header counts


def test_percentile():
    assert bench._percentile([], 0.5) is None
    assert bench._percentile([3.0], 0.99) == 3.0
    assert bench._percentile([1.0, 2.0, 3.0, 4.0], 0.5) == pytest.approx(2.5)
    assert bench._percentile(list(range(101)), 0.99) == pytest.approx(99.0)


def test_derived_alu_peaks():
    # 152 SMs x 2 FP64 FMA lanes (resp. 128 FP32) per clock x 2 flop x 2070 MHz
    assert bench.fp64_peak_gflops(2070.0) == pytest.approx(1258.56)
    assert bench.fp32_peak_gflops(2070.0) == pytest.approx(80547.84)


def test_factor_kernel_names_match_the_launch_counts():
    from paper_2609_29977_gb300 import bm as core
    # medium FP64: 4 level launches + top (whose last CTA does the root step)
    # = the factor part of the 8 launches
    assert bench._factor_kernels(64, 12, "fp64") == \
        "k_factor_level_team x4 + k_factor_top (its last CTA does the root step)"
    assert core.launches_per_step(64, 64, 12, 4) - 3 == 4 + 1
    assert bench._factor_kernels(256, 48, "fp32ir").startswith("k_level_rows_w x6 + k_top_rows_w + k_pivot_spread")
    assert bench._factor_kernels(9, 5, "fp64") == "k_factor_level x4 + k_factor_x1 + k_factor_root"
