"""Host logic of bench.py that needs no GPU: the clock sampler's reading of
nvidia-smi rows (median SM clock, the maximum, and which throttle reasons were
active), and the roofline entry's arithmetic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s


def test_clock_rows_median_max_and_reasons():
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1201.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1180.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 10, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler(rows).stop()
    assert out["sm_mhz"] == 2070.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3


def test_clock_rows_report_every_slowdown_kind():
    rows = ["0, 1500, 2070, 1300, 0x8, Active, Active, Active, Not Active"]
    out = _sampler(rows).stop()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


NCU_CSV = """==PROF== Connected
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","20.00"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","10.00"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","110.00"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","sm__inst_executed_pipe_fp64.sum","inst","2,000,000"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active","%","80.00"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","smsp__sass_thread_inst_executed_op_dadd_pred_on.sum","inst","30,000,000"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","smsp__sass_thread_inst_executed_op_dfma_pred_on.sum","inst","13,000,000"
"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7","(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","smsp__sass_thread_inst_executed_op_dmul_pred_on.sum","inst","10,000,000"
"1","1","python3","h","void k_dt(Dims, const double *, const double *, double *)","1","7","(256, 1, 1)","(10, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","3.00"
"""


def test_roofline_counts_from_ncu_csv(tmp_path):
    """The counts parser takes units into account, forms FP64 flop as 2 DFMA + DADD +
    DMUL, keeps DRAM read + write per launch and ignores kernels outside the stage."""
    from paper_2110_03732_gb300 import roofline as RL
    f = tmp_path / "counts.csv"
    f.write_text(NCU_CSV)
    kinds, names = RL.counts_from_ncu_csv(str(f), 512 * 512)
    assert list(kinds) == ["flux"]
    k = kinds["flux"]
    assert k["launches"] == 1 and k["dur_us"] == pytest.approx(110.0)
    assert k["fp64_flop"] == pytest.approx(2 * 13e6 + 30e6 + 10e6)
    assert k["dram_bytes"] == pytest.approx(30e6)
    assert k["fp64_pipe_inst"] == pytest.approx(32 * 2e6)
    assert k["fp64_flop_per_cell"] == pytest.approx(66e6 / 262144)
    # one capture per kernel kind: launches of the same ID in two files are two launches
    g = tmp_path / "counts2.csv"
    g.write_text(NCU_CSV)
    kinds2, _ = RL.counts_from_ncu_csv([str(f), str(g)], 512 * 512)
    assert kinds2["flux"]["launches"] == 2
    assert kinds2["flux"]["fp64_flop"] == pytest.approx(k["fp64_flop"])


def test_roofline_alu_entry_arithmetic_and_staleness(tmp_path, monkeypatch):
    """achieved = stored FP64 flop per launch / live mean launch time, against the
    nominal FP64 rate; a count taken on other kernel sources reports stale and no
    traffic, and changing a kernel source makes the stored counts stale."""
    import json
    import shutil
    from paper_2110_03732_gb300 import roofline as RL
    f = tmp_path / "counts.csv"
    f.write_text(NCU_CSV)
    counts = RL.build_counts(str(f))
    p = tmp_path / "roofline_counts.json"
    p.write_text(json.dumps(counts))
    c = RL.load_counts(str(p))
    assert c["stale"] is False
    ms = 0.1
    r = RL.alu_entry(c, "fp64", "flux", ms, peak_probe_tflops=1.2)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(66e6 / (ms / 1e3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / RL.FP64_PEAK_TFLOPS)
    assert r["traffic"] == pytest.approx(30e6)
    assert r["fp64_issue_frac"] == pytest.approx(32 * 2e6 / (ms / 1e3) / RL.FP64_INST_PEAK_PER_S)
    # an unknown kernel kind reports no figure rather than a made-up one
    u = RL.alu_entry(c, "fp64", "unknown", ms)
    assert u["achieved"] is None and u["frac"] is None
    # edit a copy of the kernel sources: the same stored counts are now stale
    src = tmp_path / "pkg"
    shutil.copytree(RL.HERE + "/csrc", src / "csrc")
    monkeypatch.setattr(RL, "HERE", str(src))
    assert RL.load_counts(str(p))["stale"] is False
    k = src / "csrc" / "kernels.cu"
    k.write_text(k.read_text() + "\n// edited\n")
    c2 = RL.load_counts(str(p))
    assert c2["stale"] is True
    r2 = RL.alu_entry(c2, "fp64", "flux", ms)
    assert r2["traffic"] is None and r2["counts"]["stale"] is True


def test_issue_entry_arithmetic(tmp_path):
    """The instruction-issue roofline: 32 x warp instructions per launch over the live
    launch time, against 4 schedulers x 32 lanes x 152 SMs x 2.07 GHz."""
    import json
    from paper_2110_03732_gb300 import roofline as RL
    f = tmp_path / "counts.csv"
    row = ('"0","1","python3","h","void k_flux_march<0, 0, double, 0>(Dims, FluxArgs<double>)","1","7",'
           '"(128, 1, 1)","(296, 1, 1)","0","10.3","Command line profiler metrics","smsp__inst_executed.sum",'
           '"inst","1,000,000"')
    lines = NCU_CSV.splitlines()
    f.write_text("\n".join(lines[:3] + [row] + lines[3:]) + "\n")
    counts = RL.build_counts(str(f))
    p = tmp_path / "c.json"
    p.write_text(json.dumps(counts))
    c = RL.load_counts(str(p))
    r = RL.issue_entry(c, "fp64", "flux", 0.1)
    assert RL.ISSUE_PEAK_TINST == pytest.approx(4 * 32 * 152 * 2.07e9 / 1e12)
    assert r["unit"] == "Tinst/s" and r["achieved"] == pytest.approx(32e6 / 1e-4 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / RL.ISSUE_PEAK_TINST)
    assert r["fp64_flop_frac"] == pytest.approx(RL.alu_entry(c, "fp64", "flux", 0.1)["frac"])
    assert RL.issue_entry(c, "fp64", "update", 0.1)["achieved"] is None


def test_hbm_entry_arithmetic():
    from paper_2110_03732_gb300 import roofline as RL
    r = RL.hbm_entry(None, "mixed", "flux", 0.02, 112.0 * 262144, 6780.4)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(112.0 * 262144 / 0.02e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6780.4)
    assert r["traffic"] is None
