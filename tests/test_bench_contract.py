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
