"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the contract's keys; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "M-phase particle*obs lik evals/s"
    assert line["unit"] == line["cpu_baseline"]["unit"] == line["e2e"]["unit"]
    assert line["value"] > 0 and line["value"] == line["cpu_baseline"]["value"] == line["e2e"]["value"]
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "egarch34_T20000" and line["data"] == "synthetic"


def test_roofline_operation_counts():
    """The ALU bound bench.py reports: the per-observation counts of the design
    table ((K,I) = (2,2) with gamma: 20 FP32 + 2 SFU; I = 1 has no mixture
    exponential) and the three limits at 152 SMs x 2070 MHz."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.alu_ops_per_eval(2, 2, True) == (20, 2)
    assert bench.alu_ops_per_eval(1, 1, False) == (1 + 2 + 1 + 1 + 2 + 1, 1)
    assert bench.alu_ops_per_eval(3, 4, True) == (1 + 9 + 3 + 1 + 2 + 20, 5)
    f = 152 * 2070e6
    peak, pipe = bench.alu_peak_evals(2, 2, True, 152, 2070.0)
    assert pipe == "issue" and abs(peak - f * 128 / 22) < 1e-3 * peak
    peak2, pipe2 = bench.alu_peak_evals(2, 2, True, 152, 2070.0, paired=True)
    assert pipe2 == "fp32" and abs(peak2 - f * 128 / 20) < 1e-3 * peak2
    fm, mm = bench.mala_ops_per_eval(2, 2, True)
    assert fm > 20 and mm > 2
    # measured rates replace the nominal ones pipe by pipe
    peak3, pipe3 = bench.alu_peak_evals(2, 2, True, 152, 2070.0, rates={"issue": 3.0, "ffma": 100.0})
    assert pipe3 == "issue" and abs(peak3 - f * 96 / 22) < 1e-3 * peak3
    peak4, pipe4 = bench.alu_peak_evals(3, 4, True, 152, 2070.0, rates={"ex2": 8.0})
    assert pipe4 == "mufu" and abs(peak4 - f * 8 / 5) < 1e-3 * peak4
