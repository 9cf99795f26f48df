"""Host-side arithmetic of bench.py, without a GPU: the clock record's summary (median SM clock,
maximum, throttle reasons) and the roofline entries (bound, achieved, fraction of the peak,
traffic, the dominant kernel and one entry per kernel family)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1800.0}


def _summary(tmp_path, lines):
    cs = bench.ClockSampler(0)
    os.unlink(cs.path)
    cs.path = str(tmp_path / "clocks.csv")
    cs.proc = object()  # a sampler that ran: summary() reads its file
    with open(cs.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return cs.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    row = "0, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {cap}"
    lines = [row.format(sm=s, cap="Active" if s == 1800 else "Not Active") for s in (2070, 2055, 1800, 2070, 2040)]
    s = _summary(tmp_path, lines)
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 5
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(str(tmp_path / "clocks.csv"))


def test_clock_summary_slowdowns_and_unreadable_fields(tmp_path):
    lines = ["0, 1200, 2070, 1400, 0x8, Active, Not Active, Not Active, Not Active",
             "0, [N/A], [N/A], [N/A], [N/A], Not Active, Not Active, Active, Not Active",
             "garbage line"]
    s = _summary(tmp_path, lines)
    assert s["sm_mhz"] == 1200 and s["sm_max_mhz"] == 2070 and s["samples"] == 2
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s = _summary(tmp_path, ["0, [N/A], [N/A], 1, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["sm_mhz"] is None and s["sm_max_mhz"] is None and s["reasons"] == []
    assert _summary(tmp_path, [])["reasons"] == ["no samples"]


def test_clock_summary_without_nvidia_smi():
    cs = bench.ClockSampler(0)
    assert os.path.exists(cs.path)
    assert cs.summary()["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(cs.path)


@pytest.fixture
def fixed_peaks(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (dict(PEAKS), "measured"))
    monkeypatch.setattr(bench, "fp32_peak", lambda dev, clocks: (80.0, "derived"))


def test_roof_entry_hbm_bound(fixed_peaks):
    # 10 launches moving 1 GB in all within 0.25 ms: 4000 GB/s of 7000
    e = bench.roof_entry("cd_spectrum_kernel", [10, 0.25, 1e9, 1e9], None, None)
    assert e["bound"] == "hbm" and e["unit"] == "GB/s" and e["peak"] == 7000.0
    assert e["achieved"] == pytest.approx(4000.0) and e["frac"] == pytest.approx(4000.0 / 7000.0)
    assert e["avg_launch_ms"] == pytest.approx(0.025) and e["algorithmic_bytes_per_launch"] == pytest.approx(1e8)
    assert e["traffic"] == bench.NCU_TRAFFIC["cd_spectrum_kernel"]


def test_roof_entry_alu_and_tensor_bound(fixed_peaks):
    # FP32 SIMT work: 40 TFLOP in 1 s at an 80 TFLOP/s peak, bytes negligible
    e = bench.roof_entry("cd_apply_kernel", [4, 1000.0, 40e12, 1e6], None, None)
    assert e["bound"] == "alu" and e["achieved"] == pytest.approx(40.0) and e["frac"] == pytest.approx(0.5)
    # TF32x3 GEMM: the sustained BF16 rate x the nominal TF32 : BF16 ratio / 3
    e = bench.roof_entry("umma_gemm_kernel<true>", [1, 1000.0, 100e12, 1e6], None, None)
    peak = 1800.0 * bench.TF32_PER_BF16 / 3.0
    assert e["bound"] == "tensor" and e["peak"] == pytest.approx(peak)
    assert e["frac"] == pytest.approx(100.0 / peak)
    e = bench.roof_entry("umma_gemm_kernel<false>", [1, 1000.0, 900e12, 1e6], None, None)
    assert e["peak"] == 1800.0 and e["frac"] == pytest.approx(0.5)
    # a kernel absent from the ncu table reports its traffic as null; no work: latency
    e = bench.roof_entry("cd_select_kernel", [3, 0.1, 0.0, 0.0], None, None)
    assert e["bound"] == "latency" and e["frac"] is None and e["traffic"] is None


def test_roofline_dominant_kernel_and_families(fixed_peaks):
    trace = {  # label: launches, ms, flops, bytes
        "cd_apply_col": (2, 0.20, 1e11, 2e8), "cd_apply_row": (2, 0.20, 1e11, 2e8),
        "cd_spectrum": (2, 0.15, 1e9, 4e8), "cd_residual_direct": (3, 0.05, 1e9, 3e8),
        "umma_gemm_tf32x3": (6, 0.30, 4e12, 1e8), "ft_t2": (1, 0.02, 1e9, 1e8),
    }
    r = bench.roofline(trace, None, None)
    assert r["kernel"] == "cd_apply_kernel" and r["launches"] == 4  # both apply labels merge: 0.40 ms
    assert r["share_of_step"] == pytest.approx(0.40 / 0.92)
    fams = r["families"]
    assert set(fams) == {"spectral_apply", "fft", "tcgen05_gemm", "sparsifier_apply"}
    assert fams["fft"]["kernel"] == "cd_spectrum_kernel"  # the family's longest kernel
    assert fams["tcgen05_gemm"]["bound"] == "tensor"


def test_clock_sampler_without_the_tool_reports_and_cleans_up(monkeypatch):
    def no_tool(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(bench.subprocess, "Popen", no_tool)
    with bench.ClockSampler(0) as clk:
        pass
    assert clk.f.closed
    assert clk.summary()["reasons"] == ["nvidia-smi unavailable"] and not os.path.exists(clk.path)


def test_clock_rejection_rules():
    ok = {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert bench.clock_rejection(ok) == []
    assert bench.clock_rejection(dict(ok, reasons=["sw_power_cap"])) == []
    assert bench.clock_rejection(dict(ok, sm_mhz=1500.0, reasons=["sw_power_cap"])) == []  # capped, kept
    assert bench.clock_rejection(dict(ok, reasons=["sw_power_cap", "hw_slowdown"])) == ["hw_slowdown"]
    assert bench.clock_rejection(dict(ok, reasons=["sw_thermal_slowdown"])) == ["sw_thermal_slowdown"]
    stuck = bench.clock_rejection(dict(ok, sm_mhz=1200.0))
    assert len(stuck) == 1 and "no reason" in stuck[0]
    assert bench.clock_rejection({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}) == []
    assert bench.clock_rejection(None) == []
