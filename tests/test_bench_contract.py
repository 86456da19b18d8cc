"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON
line with the keys and units the GPU arm uses; it needs no GPU, so it runs
here on a one-step sample."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    sys.path.insert(0, ROOT)
    import bench

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD and tuple(d["config"]["cases"]) == bench.CASES
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == bench.UNIT
    assert cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == bench.UNIT
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_clock_sampler_parses_nvidia_smi_lines():
    """The clocks object of the bench line: median SM clock under load, the
    highest max clock seen and every throttle reason reported Active."""
    sys.path.insert(0, ROOT)
    import bench

    s = bench.ClockSampler(0)
    s.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    s.lines = [
        "1980, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2055, 2070, 1050.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    c = s.stop()
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.lines = ["1500, 2070, 1200.0, 0x20, Not Active, Active, Not Active, Not Active"]
    assert s.stop()["reasons"] == ["hw_thermal_slowdown"]
    s.lines = []
    assert s.stop() is None


def test_roofline_splits_the_persistent_launch_by_phase():
    """The dominant kernel's roofline: survey-unit pair work against the FP32
    issue rate, the two-pipe fraction (double-float pairs at the FP32 rate
    plus the G rows' FP64 multiply-adds at the FP64 rate, over the launch's
    time), and the sweep (a2) and growth (a4) apart over their phases' time."""
    import bench

    st = dict(persist_ms=10000.0, persist_launches=2, sweep_pairs_useful=4e10, newton_ms=500.0,
              newton_launches=3, newton_pairs_useful=1e9, vol_ms=100.0, vol_launches=3, vol_pairs_useful=4e9,
              sweep_ms=0.0, sweep_launches=0, persist_grow_fma=2e12,
              persist_phase_ms=[1500.0, 1500.0, 0.0, 0.0, 600.0, 400.0, 5000.0, 1000.0])
    sms, clk = 152, 2.07e9
    fp32_peak = sms * 128 * clk
    fp64_fma = sms * 2 * clk
    r = bench.roofline_of([st], 3, sms, clk, True)
    assert r["kernel"].startswith("k_greedy_persist")
    assert abs(r["frac"] - 4e10 * 16 / 10.0 / fp32_peak) < 1e-12
    want = (4e10 * 284 / fp32_peak + 2e12 / fp64_fma) / 10.0
    assert abs(r["persist_pipes"]["frac"] - round(want, 5)) < 1e-5
    a2, a4 = r["persist_by_phase"]["a2_sweep"], r["persist_by_phase"]["a4_grow"]
    assert a2["s"] == 3.0 and a4["s"] == 7.0 and a4["g_rows_s"] == 6.0
    assert abs(a2["frac"] - round(4e10 * 16 / 3.0 / fp32_peak, 5)) < 1e-5
    assert abs(a4["g_rows_frac"] - round(2e12 / 6.0 / fp64_fma, 5)) < 1e-5
    # FP64 mode: the sweep's pairs run on the FP64 pipe
    r = bench.roofline_of([st], 3, sms, clk, False)
    a2 = r["persist_by_phase"]["a2_sweep"]
    assert a2["frac_df_ops"] is None and abs(a2["frac"] - round(4e10 * 16 / 3.0 / fp64_fma, 5)) < 1e-5
    assert r["persist_pipes"]["frac"] is None
