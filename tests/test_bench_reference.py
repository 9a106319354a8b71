"""The reference arm of bench.py (the CPU oracle, no GPU): one JSON line with the fields the
benchmark contract asks for, on a small oracle sample so that it runs in seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                        "--sample-n", "200,300"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "n=300" in d["cpu_baseline"]["sample"]
    # one step per size (n = 300, then 200): the law is a fit over both measured points
    fit = d["cpu_baseline"]["fit"]
    assert fit["fitted"] and sorted(q[0] for q in fit["points"]) == [200, 300]
    assert abs(fit["coef"] * 300 ** fit["exponent"] - [q[1] for q in fit["points"] if q[0] == 300][0]) <= \
        1e-6 * fit["coef"] * 300 ** fit["exponent"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("RT-shaped QP")
