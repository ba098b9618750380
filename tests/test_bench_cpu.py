"""The reference arm of bench.py (the FP64 oracle on the host cores) prints the
contract's JSON line: same metric, unit and workload description as the GPU arm,
impl = "reference", a cpu_baseline object and a host-only e2e object."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "particle-steps/s" and d["higher_is_better"] is True
    assert d["metric"].startswith("particle-steps/s")
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"].startswith("batched_mixed: 1024 samples, 4107..32737 particles each")
    b = d["cpu_baseline"]
    assert b["kind"] == "oracle" and b["cores"] >= 1 and b["value"] == d["value"] and b["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_measured_pipe_peaks_are_read_from_the_committed_summary():
    import bench
    from paper_2205_04979_gb300 import peaks
    rec = peaks.load(bench.PEAKS_FILE)
    assert rec is not None and rec["sms"] > 0 and rec["clocks"]["sm_mhz"] > 0
    fp32, _, mix32 = bench.pipe_peak(True, True)
    fp64, _, mix64 = bench.pipe_peak(False, False)
    assert fp32 == rec["kernels"]["ffma2"]["flops_per_s"] / 1e12
    assert fp64 == rec["kernels"]["dfma"]["flops_per_s"] / 1e12
    # the Newton-pair mix: 16 pipe operations for 24 flops
    assert abs(mix32["peak"] - 2 * rec["kernels"]["ffma2"]["lane_ops_per_s"] * 1.5 / 1e12) < 1e-9
    assert mix64 is None


def test_reference_arm_of_the_low_fidelity_workload():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "lf_eulerian", "--samples", "24", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "evaluations/s" and d["value"] > 0
    assert d["config"]["workload"] == "lf_eulerian: 24 samples x 10 St+ classes"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
