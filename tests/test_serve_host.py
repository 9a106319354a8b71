"""Host logic of the serving loop (no GPU): request stream, per-step costs, admission under
max_inflight and the HBM ledger, chains keeping their slot, results routed per request.

The solver handle is replaced by a host-only fake whose "solution" is a fixed function of
the costs it was given, so the scheduler's routing can be checked exactly."""
import time

import numpy as np
import pytest

from paper_2405_03584_gb300 import workloads as W
from paper_2405_03584_gb300 import serve


def test_serving_stream_statistics():
    reqs = W.serving_stream(horizon=60.0, lam=20.0, chain_frac=0.3, chain_len=20, n_plans=64, seed=4)
    assert reqs == W.serving_stream(horizon=60.0, lam=20.0, chain_frac=0.3, chain_len=20, n_plans=64, seed=4)
    n = len(reqs)
    assert abs(n - 1200) < 4 * np.sqrt(1200)           # Poisson count, mean lam * horizon
    ts = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(ts) > 0) and ts[-1] < 60.0
    gaps = np.diff(np.concatenate([[0.0], ts]))
    assert abs(gaps.mean() - 1 / 20.0) < 4 * (1 / 20.0) / np.sqrt(n)
    chains = sum(r["steps"] == 20 for r in reqs)
    assert all(r["steps"] in (1, 20) for r in reqs)
    assert abs(chains / n - 0.3) < 4 * np.sqrt(0.21 / n)
    assert {r["plan"] for r in reqs} <= set(range(64))


def test_request_costs_regenerate_any_step():
    p = W.rt_qp(n=40, seed=2)
    req = dict(seed=1234)
    prev, seq = None, []
    for _ in range(4):
        prev = W.request_costs(p, req, prev)
        seq.append(prev)
    assert [s[2] for s in seq] == [0, 1, 2, 3]
    # step 0 is a 1% perturbation of the plan's costs, step k+1 of step k
    assert 0 < np.max(np.abs(seq[0][0] / p["w"] - 1)) < 0.06
    nz = seq[1][1] != 0
    assert nz.any() and np.all(seq[2][1][~nz] == 0)
    assert 0 < np.max(np.abs(seq[2][1][nz] / seq[1][1][nz] - 1)) < 0.06
    again = W.request_costs(p, req, seq[1])
    assert np.array_equal(again[0], seq[2][0]) and np.array_equal(again[1], seq[2][1])
    assert np.all(seq[3][0] > 0)


class FakeSolver:
    """Stands in for ipm.Solver: a solve lasts ``dt`` seconds; x = c + sum(f_w)."""
    live = 0
    max_live = 0
    dt = 0.003

    def __init__(self, **opts):
        self.t_end = None
        self.closed = False

    def set_qp_rt(self, p, stream=None):
        self.p, self.n, self.matrix = p, p["n"], 1000 * p["n"]
        return self

    def share_qp(self, src, stream=None):
        self.p, self.n, self.matrix = src.p, src.n, src.matrix
        return self

    def device_bytes(self):
        return dict(matrix=self.matrix, state=10 * self.n, matrix_refs=1)

    def update_costs(self, f_w=None, c=None, stream=None):
        assert self.t_end is None and not self.closed
        self.w, self.c = f_w, c

    def solve_async(self, warm=False, stream=None):
        assert self.t_end is None
        FakeSolver.live += 1
        FakeSolver.max_live = max(FakeSolver.max_live, FakeSolver.live)
        self.warm = warm
        self.t_end = time.perf_counter() + self.dt

    def done(self):
        return time.perf_counter() >= self.t_end

    def wait(self):
        FakeSolver.live -= 1
        self.t_end = None
        return 0

    def get(self, stream=None):
        info = dict(ipm_iters=5 if self.warm else 10, cg_iters=50, rel_kkt=1e-9, primal_obj=0.0)
        return dict(x=self.c + self.w.sum(), info=info)

    def close(self):
        self.closed = True


@pytest.fixture
def fake_server(monkeypatch):
    monkeypatch.setattr(serve.Server, "solver_cls", FakeSolver)
    monkeypatch.setattr(serve.Server, "stream_factory", staticmethod(lambda: None))
    FakeSolver.live = FakeSolver.max_live = 0
    return serve.Server


def test_scheduler_routes_costs_and_respects_limits(fake_server):
    plans = [W.rt_qp(n=n, seed=k) for k, n in enumerate((30, 50, 70))]
    reqs = W.serving_stream(horizon=0.15, lam=300.0, chain_frac=0.4, chain_len=4, n_plans=3, seed=9)
    assert any(r["steps"] == 4 for r in reqs) and any(r["steps"] == 1 for r in reqs)
    srv = fake_server(plans, budget_bytes=1e12, max_inflight=3, keep_x=True)
    plan_bytes = srv.used
    # room for two extra slot states beyond the plans' own handles
    srv.budget = plan_bytes + 2 * 10 * 70
    qrec, rrec = srv.run(reqs)
    assert len(qrec) == sum(r["steps"] for r in reqs)
    assert FakeSolver.max_live <= 3 and srv.stats["max_inflight_seen"] <= 3
    assert srv.stats["ledger_peak_bytes"] <= srv.budget
    by = {(r["rid"], r["step"]): r for r in qrec}
    for r in reqs:
        prev = None
        for k in range(r["steps"]):
            prev = W.request_costs(plans[r["plan"]], r, prev)
            rec = by[(r["rid"], k)]
            assert np.array_equal(rec["x"], prev[1] + prev[0].sum())
            assert rec["warm"] == (k > 0)
            assert rec["latency"] >= FakeSolver.dt * 0.9
            if k:
                assert rec["t_release"] == by[(r["rid"], k - 1)]["t_done"]
            else:
                assert rec["t_release"] == r["t"]
    for rr in rrec:
        assert rr["latency"] >= rr["steps"] * FakeSolver.dt * 0.9
    s = serve.latency_summary(qrec, rrec, 0.15, srv.stats["busy_s"])
    assert s["qps"] == len(qrec) and s["p99_ms"] >= s["p50_ms"] > 0
    assert s["ipm_iters_warm"] == 5 and s["ipm_iters_cold"] == 10
    srv.close()


def test_ledger_frees_idle_slots_of_other_plans(fake_server):
    plans = [W.rt_qp(n=n, seed=k) for k, n in enumerate((40, 40))]
    srv = fake_server(plans, budget_bytes=1e12, max_inflight=4)
    srv.budget = srv.used + 10 * 40          # one extra slot state fits
    extra = srv._new_slot(0)
    assert extra is not None and srv.used == srv.budget
    srv.idle[0].append(extra)
    assert srv._new_slot(1) is not None       # frees plan 0's idle shared slot first
    assert extra.solver.closed and srv.slots_freed == 1
    assert srv._new_slot(1) is None           # plan handles are never freed; no room left
    srv.close()


def test_plans_over_budget_rejected(fake_server):
    plans = [W.rt_qp(n=40, seed=1)]
    with pytest.raises(MemoryError):
        fake_server(plans, budget_bytes=1000)
