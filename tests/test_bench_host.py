"""Host logic of bench.py that needs no GPU: the summary of the clock
samples taken during the timed region (median SM clock, maximum clock,
throttle reasons that reject a run), the FP32 work per unit of the roofline,
and the DRAM traffic record, which is used only while the step kernel's
sources are the captured ones."""
import json

import bench


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 812.35, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_clock_summary_median_max_and_reasons():
    lines = [_row(2070, 2070), _row(2055, 2070), _row(2070, 2070, cap="Active"), _row(1980, 2070)]
    c = bench.summarize_clocks(lines)
    assert c == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}


def test_clock_summary_reports_every_throttle_reason():
    lines = [_row(1500, 2070, hw="Active"), _row(1400, 2070, hwt="Active"), _row(1450, 2070, swt="Active")]
    c = bench.summarize_clocks(lines)
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1450.0


def test_clock_summary_skips_unreadable_fields_and_short_lines():
    lines = ["garbage\n", _row("[N/A]", 2070), _row(2070, "[N/A]"), "0, 2070\n"]
    c = bench.summarize_clocks(lines)
    assert c["samples"] == 2 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert bench.summarize_clocks([]) is None and bench.summarize_clocks(["x\n"]) is None


def test_flops_per_unit():
    # 2 d^2 + 13 d + 20 (Euler, locate, centring, y/z evaluation, clamps,
    # driver, response) + 18 per normal (degree-9 polynomial), d normals
    assert [bench.flops_per_path_step(d) for d in (1, 2, 4, 6)] == [53.0, 90.0, 176.0, 278.0]
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9


def test_traffic_record_needs_the_captured_sources(tmp_path, monkeypatch):
    rec = {"records": [{"workload": "w", "control": False, "kernel_source_sha256": bench.kernel_source_hash(),
                        "dram_bytes_per_launch": 123.0}]}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "step_kernel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["records"][0]["kernel_source_sha256"])
    assert bench.recorded_traffic("w", False) == 123.0
    assert bench.recorded_traffic("w", True) is None
    assert bench.recorded_traffic("other", False) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.recorded_traffic("w", False) is None


def test_oracle_time_extrapolation():
    # per-stratum fit times a + b (N - i) measured at three steps (wall time of
    # n fits), summed over all K strata and N steps: exact for that model
    from paper_2407_21085_gb300 import workloads as W
    w = W.cfg2(C=8, N=10, M=64)
    a, b = 0.002, 0.0005
    fits = [(i, n, n * (a + b * (w.N - i)), 0) for i, n in ((0, 4), (5, 4), (9, 16))]
    want = sum(w.K * (a + b * (w.N - i)) for i in range(w.N))
    assert abs(bench.extrapolate_full(w, fits) - want) < 1e-9 * want
    # the sampled steps are 0, N/2 and N-1, with more strata at the cheap last step
    plan = bench.oracle_plan(w, 8, single=False)
    assert [i for i, _ in plan] == [0, w.N // 2, w.N - 1] and plan[2][1] > plan[0][1]
    assert all(n == 1 for _, n in bench.oracle_plan(w, 1, single=True)[:2])


def test_z_evaluation_share_of_the_flop_count():
    # the z row's multiply-adds d (d + 1) and its d clamps, inside 2 d^2 + 13 d + 20
    assert [bench.z_eval_flops(d) for d in (1, 2, 6)] == [6.0, 16.0, 96.0]
    assert bench.flops_per_path_step(6) - bench.z_eval_flops(6) == 182.0
