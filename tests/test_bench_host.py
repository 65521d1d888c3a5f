"""bench.py's host logic (no GPU): the reference arm's JSON line (the CPU
oracle timed on a bounded sample of the workload) and the parsing of the
nvidia-smi clock samples taken during the timed region."""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "grover30_qft_sweep_c128"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.lines = list(lines)
    return cs.stop()


def test_clock_samples_median_and_reasons():
    # index, clocks.sm, clocks.max.sm, power, active mask, hw_slowdown,
    # hw_thermal, sw_thermal, sw_power_cap (the query order bench.py uses)
    r = _sampler(["0, 2070, 2070, 910.2, 0x0, Not Active, Not Active, Not Active, Not Active",
                  "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                  "0, 2070, 2070, 905.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    r = _sampler(["0, 1500, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active", "garbage", "0, [N/A], 2070"])
    assert r["samples"] == 1 and r["sm_mhz"] == 1500.0
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    import bench
    cs = bench.ClockSampler(0)  # never started: no process
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
