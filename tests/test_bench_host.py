"""Host logic of the benchmark on the CPU: the clock summary of the sampled
nvidia-smi rows, the per-kernel roofline arithmetic, the choice of the
dominant kernel and the algorithmic work counts the roofline divides."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %s, %s, 812.40, 0x0000000000000000, %s, %s, %s, %s\n" % (sm, mx, hw, hwt, swt, cap)


def test_clock_summary_median_max_and_no_reasons():
    c = bench.summarize_clocks([_row(2070, 2070), _row(2055, 2070), _row(2070, 2070)])
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070 and c["reasons"] == [] and c["samples"] == 3


def test_clock_summary_reports_each_active_reason_once():
    rows = [_row(1980, 2070, cap="Active"), _row(2070, 2070), _row(1900, 2070, cap="Active", hwt="Active")]
    c = bench.summarize_clocks(rows)
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert c["sm_mhz"] == 1980


def test_clock_summary_skips_short_rows_and_unavailable_clocks():
    rows = ["garbage\n", "0, [N/A], [N/A], 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
            _row(2070, 2070)]
    c = bench.summarize_clocks(rows)
    assert c["samples"] == 2 and c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070
    assert bench.summarize_clocks([])["reasons"] == ["no samples"]


class _WL:
    def __init__(self, dof, p, n_comp, n1):
        self.dof, self.p, self.n_comp, self.vel_n = dof, p, n_comp, (n1, n1, n1)


def _result(stage_ms, q_ms, launches, iters):
    return {"prof": {"stage": (stage_ms * launches, launches), "qprime": (q_ms * launches, launches)},
            "newton": {"mean_iters": iters}}


def test_mixed_roofline_is_algorithmic_bytes_over_event_time():
    wl = _WL(3.62e9, 3, 1, 24)
    peaks = {"hbm_gbs": 6689.8, "fp32_fma": 78.5e12, "fp64_fma": 1.256e12}
    rl = bench.kernel_rooflines(wl, _result(21.4, 7.9, 9, 0.0), peaks, "mixed")
    st = rl["stage"]
    assert st["bound"] == "hbm" and st["unit"] == "GB/s"
    # 10.67 B per DOF (F read + write, f^n in two of three stages, FP32) in 21.4 ms
    assert st["achieved"] == pytest.approx(3.62e9 * 4 * 8 / 3 / 21.4e-3 / 1e9)
    assert st["achieved"] == pytest.approx(1804, rel=1e-3)
    assert st["frac"] == pytest.approx(st["achieved"] / 6689.8)
    assert st["traffic"] is None
    d = bench.dominant_roofline(rl)
    assert d["kernel"] == "stage" and "MEASURED_PEAKS" in d["peak_source"]


def test_fp64_roofline_counts_flops_and_evaluations():
    wl = _WL(3.62e9, 3, 1, 24)
    peaks = {"hbm_gbs": 6689.8, "fp32_fma": 78.5e12, "fp64_fma": 1.256e12}
    rl = bench.kernel_rooflines(wl, _result(384.0, 246.0, 3, 2.0), peaks, "fp64")
    assert rl["stage"]["achieved"] == pytest.approx(3.62e9 * 100.25 / 0.384 / 1e12)
    assert rl["qprime"]["achieved"] == pytest.approx(3.62e9 * 3.0 * (12 + 109 / 24) / 0.246 / 1e12)
    assert rl["stage"]["frac"] == pytest.approx(rl["stage"]["achieved"] / 1.256)
    assert bench.dominant_roofline(rl)["kernel"] == "stage"
    # the longer kernel dominates whichever it is
    rl = bench.kernel_rooflines(wl, _result(100.0, 246.0, 3, 2.0), peaks, "fp64")
    assert bench.dominant_roofline(rl)["kernel"] == "qprime"


def test_algorithmic_work_counts():
    # FR 6(p+1) + 5 + 12 + 9/(p+1) + 6 per component, equilibrium/source/RK 26 + 3, epilogue 22
    assert bench.stage_flops_per_dof(3, 1) == pytest.approx(100.25)
    assert bench.stage_flops_per_dof(1, 1) == pytest.approx(6 * 2 + 5 + 12 + 4.5 + 6 + 29 + 22)
    # G adds a second FR, 4 source flops and 2 epilogue flops
    assert bench.stage_flops_per_dof(2, 2) - bench.stage_flops_per_dof(2, 1) == pytest.approx(6 * 3 + 5 + 12 + 3 + 6 + 6)
    assert bench.stage_bytes_per_dof(1, 4) == pytest.approx(32 / 3)
    assert bench.stage_bytes_per_dof(2, 8) == pytest.approx(128 / 3)
    assert bench.job_throughput(1, 3.62e9, 3, 87.9 * 3) == pytest.approx(3.62e9 * 3 / (87.9e-3))


def test_drift_is_a_conservation_measure_only_on_closed_meshes():
    from paper_2312_06567_gb300 import workloads as W
    assert bench.drift_is_conservation(W.taylor_green_box())            # periodic box
    assert bench.drift_is_conservation(W.periodic_sine_box())
    assert not bench.drift_is_conservation(W.normal_shock_tube())       # Dirichlet x-ends
    assert not bench.drift_is_conservation(W.sphere_ogrid(n=(2, 4, 4), vel_n=(6, 6, 6)))  # wall, farfield
    box = W.normal_shock_tube().replace(dirichlet={})
    assert bench.drift_is_conservation(box.replace(closed=((0, -1), (0, 1))))
    assert not bench.drift_is_conservation(box.replace(specular=((0, -1), (0, 1))))
    assert not bench.drift_is_conservation(box.replace(closed=((0, -1),), specular=((0, 1),)))


def _fake_form(stage_ms, q_ms, iters, learned=False, e2e=None):
    """What run_ours records per form, for one profiled step (3 stages)."""
    prof = {"moments": (0.0, 0), "qprime": (3 * q_ms, 3), "stage": (3 * stage_ms, 3), "other": (0.0, 0),
            "wall": (0.0, 0)}
    newton = dict(mean_iters=iters, max_iters=int(iters), max_residual=1e-7)
    if learned:
        newton["guess_fallbacks"] = 0
        newton["training"] = {"seconds": 0.5, "epochs": 8}
    return dict(ms=3 * (3 * stage_ms + 3 * q_ms), status="BGK_OK", prof=prof,
                clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
                newton=newton, e2e=e2e, drift=3e-11, stage_kernel={"variant": "line", "depth": 2, "ms_per_stage": stage_ms},
                diagnostics=None)


def test_json_line_carries_the_contract_keys():
    """compose_line on recorded-looking results: the headline form, the
    contract keys, the dominant kernel's roofline with the measured traffic,
    the other forms nested, and a line that serialises as JSON."""
    import argparse
    import json
    from paper_2312_06567_gb300 import workloads as W
    wl = W.taylor_green_box()
    e2e = {"value": 2.1e10, "unit": bench.UNIT, "h2d_bytes_per_step": 14495514624, "d2h_bytes_per_step": 14495514624}
    results = {"fp64": _fake_form(383.0, 247.0, 2.0),
               "mixed": _fake_form(21.5, 11.6, 1.0),
               "mixed_learned": _fake_form(21.4, 7.9, 0.0, learned=True, e2e=e2e)}
    peaks = {"fp64_fma": 1.256e12, "fp32_fma": 78.5e12, "hbm_gbs": 6689.8}
    args = argparse.Namespace(steps=3, warmup=3, no_graphs=False)
    line = bench.compose_line(args, wl, results, peaks, 1)
    json.dumps(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "clocks", "e2e", "gpu_launches", "roofline"):
        assert k in line, k
    assert line["config"]["form"] == "mixed_learned" and line["config"]["workload"] == wl.name
    assert line["value"] == pytest.approx(wl.dof * 3 / (3 * (3 * 21.4 + 3 * 7.9) / 3 * 1e-3))
    assert line["gpu_launches"] == 6 * 3 and line["e2e"] == e2e
    assert line["drift_is_conservation"] is True
    rl = line["roofline"]
    assert rl["kernel"] == "stage" and rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert rl["frac"] == pytest.approx(rl["achieved"] / 6689.8)
    assert rl["traffic"] == pytest.approx(11.42 * wl.dof)      # ncu traffic of the line kernel, per launch
    assert set(line) >= {"mixed", "fp64"} and line["fp64"]["value"] < line["mixed"]["value"]
    assert line["fp64"]["roofline_kernels"]["stage"]["unit"] == "TFLOP/s"


def test_clock_sampler_without_nvidia_smi_reports_it(monkeypatch):
    """No nvidia-smi on the host: the sampler records that instead of failing."""
    def missing(*a, **k):
        raise OSError("nvidia-smi not found")
    monkeypatch.setattr(bench.subprocess, "Popen", missing)
    cs = bench.ClockSampler(0)
    cs.start()
    c = cs.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(cs.out.name)                  # no temporary file left behind


def test_clock_sampler_reads_a_running_nvidia_smi(tmp_path, monkeypatch):
    """A stand-in nvidia-smi on PATH printing rows every 50 ms: the sampler
    starts it, stops it and summarises what it printed."""
    import stat
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nwhile true; do\n"
                    "  echo '0, 2070, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
                    "  sleep 0.05\ndone\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    cs = bench.ClockSampler(0)
    cs.start()
    time.sleep(0.4)
    c = cs.stop()
    assert c["samples"] >= 2 and c["sm_mhz"] == 2070 and c["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(cs.out.name)


def test_all_cores_oracle_timing_runs_spawned_processes():
    """The all-cores leg of the CPU baseline: spawned processes (never forked
    after CUDA work), each running the unchanged oracle on its own sample."""
    r = bench.cpu_baseline_all_cores("sine_box", 1, procs=2)
    assert r["processes"] == 2 and r["value"] > 0 and r["cores"] > 0.5
    assert r["unit"] == bench.UNIT and "2 processes" in r["sample"]


def test_reference_arm_line_carries_the_contract_keys(monkeypatch, capsys):
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the metric, its cpu_baseline description and a zero-copy e2e."""
    import json
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "sine_box",
                                      "--steps", "1", "--warmup", "0"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 1 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] > 0 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOADS["sine_box"]().name
