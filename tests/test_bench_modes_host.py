"""Every mode of bench.py run on the CPU with the CUDA calls and the solver handle replaced by
stand-ins (in a child process, so that the stand-in torch never meets the other tests): the
host code of each mode runs to its JSON line and the line has the fields the benchmark
contract names.  The numbers are the stand-ins' and mean nothing; the GPU runs give the real
ones."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r'''
import contextlib, io, json, sys, types
import numpy as np
sys.path.insert(0, ROOT)


class Ev:
    def __init__(self, **k): pass
    def record(self, s=None): pass
    def elapsed_time(self, o): return 10.0


class Pinned:
    def __init__(self, a): self.a = a
    def pin_memory(self): return self
    def numpy(self): return self.a


torch = types.ModuleType("torch")
torch.cuda = types.SimpleNamespace(set_device=lambda d: None, current_device=lambda: 0, synchronize=lambda: None,
                                   current_stream=lambda: object(), Event=Ev, is_available=lambda: True)
torch.from_numpy = lambda a: Pinned(a)
dist = types.ModuleType("torch.distributed")
dist.is_available = lambda: True
dist.is_initialized = lambda: False
dist.get_world_size = lambda: 1
torch.distributed = dist
sys.modules["torch"] = torch
sys.modules["torch.distributed"] = dist

from paper_2405_03584_gb300 import build, ipm
build.build = lambda *a, **k: None


class StandInSolver:
    def __init__(self, **opts): self.n = self.m = 0
    def __enter__(self): return self
    def __exit__(self, *a): pass
    def close(self): pass
    def set_qp(self, n, m, *a, **k): self.n, self.m = n, m; return self
    def set_qp_rt(self, p): self.n, self.m = p["n"], p["m"]; return self
    def set_qp_bfgs(self, p): self.n, self.m = p["n"], p["m"]; return self
    def set_qp_dense(self, H, c, A, b, l=None, u=None, **k): self.n, self.m = len(c), len(b); return self
    def set_lowrank(self, *a, **k): pass
    def update_costs(self, *a, **k): pass
    def solve(self, warm=False, stream=None): return 0
    def sizes(self): return dict(n=self.n, m=self.m, m_rows=self.m)
    def get(self):
        info = dict(status=0, ipm_iters=20, cg_iters=200, max_cg_step=10, max_stiff_rows=5, precond=1, rel_kkt=1e-7,
                    kernel_launches=1000, lanes_rows=8, lanes_cols=16, refine_passes=0, fallback_steps=0,
                    op_arith=1, rows_runs=1, cols_gap=0)
        return dict(x=np.zeros(self.n), y=np.zeros(self.m), zl=np.zeros(self.n), zu=np.zeros(self.n),
                    s=np.zeros(self.m), info=info)
    def profile_operator(self, reps=20):
        return dict(ms_rows=0.13, ms_cols=0.12, bytes_rows=6e8, bytes_cols=6e8, flops_rows=1e8, flops_cols=1e8)


class StandInBatch:
    def __init__(self, solvers): self.k = len(solvers)
    def solve(self): return [0] * self.k
    def close(self): pass


ipm.Solver = StandInSolver
ipm.Batch = StandInBatch
import bench
bench._serve_once = lambda *a, **k: (dict(solves_per_s=10.0, p50_ms=1.0, p99_ms=2.0, max_rel_kkt=1e-7), [])


def run(argv):
    sys.argv = ["bench.py"] + argv
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main()
    lines = [l for l in buf.getvalue().splitlines() if l.startswith("{")]
    assert rc == 0 and len(lines) == 1, (argv, rc, buf.getvalue()[-500:])
    return json.loads(lines[0])


out = {}
out["default"] = run(["--steps", "2", "--warmup", "3", "--sample-n", "300"])
out["two_sided"] = run(["--two-sided", "--steps", "2", "--warmup", "3"])
out["bfgs"] = run(["--bfgs", "vmat", "--steps", "2", "--warmup", "3"])
out["dense"] = run(["--dense", "--steps", "2", "--warmup", "3"])
out["serve"] = run(["--serve", "--serve-horizon", "1", "--warmup", "3", "--batch-scale", "0.01"])
out["batch"] = run(["--batch", "--batch-count", "4", "--batch-scale", "0.02", "--steps", "2", "--warmup", "3"])
out["sqp"] = run(["--sqp", "--sqp-n", "300", "--sqp-iters", "3", "--warmup", "3"])
print("RESULT " + json.dumps(out))
'''


def test_every_bench_mode_runs_to_its_json_line(tmp_path):
    script = tmp_path / "harness.py"
    script.write_text("ROOT = %r\n" % ROOT + HARNESS)
    r = subprocess.run([sys.executable, str(script)], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1][len("RESULT "):])
    d = res["default"]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks"):
        assert key in d, key
    assert d["config"]["workload"].startswith("RT-shaped QP") and d["gpu_launches"] > 0
    assert set(d["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert d["cpu_baseline"]["kind"] == "oracle" and "n=300" in d["cpu_baseline"]["sample"]
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert res["two_sided"]["two_sided"]["m_rows"] > 0 and "one_sided" in res["two_sided"]
    assert res["bfgs"]["solve"]["rel_kkt_device"] == 1e-7 and "roofline" in res["bfgs"]
    assert res["dense"]["cpu_baseline"]["kind"] == "oracle"
    assert res["serve"]["speedup_solves_per_s"] == 1.0
    assert res["batch"]["config"]["count"] == 4
    assert res["sqp"]["warm"]["converged"]
    # every mode records the SM clocks of its timed region (None here: no nvidia-smi)
    for mode, line in res.items():
        assert "clocks" in line, mode
    assert d["e2e"]["steps"] == 5 and "cold_autotune" in d["e2e"]
    # outside the CPU-baseline legs no mode reports anything computed by oracle/
    assert not any("checker" in k for m in res.values() for k in m)
