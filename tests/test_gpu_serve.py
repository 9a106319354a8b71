"""Serving on the GPU: shared plans, per-request costs, warm-started chains, and the check
that every result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2405_03584_gb300 import ipm
from paper_2405_03584_gb300 import serve
from paper_2405_03584_gb300 import workloads as W
from oracle import kkt_check
from oracle import ipm as O

pytestmark = pytest.mark.gpu


def _rt_with(p, w, c):
    q = dict(p)
    q["w"], q["c"] = w, c
    return q


def _obj_close(p, obj, rel=1e-6):
    qp = O.from_rt(p)
    ref, info = O.solve(qp, tol=1e-10)
    assert info.status == "optimal"
    f = O.objective(qp, ref.x)
    return abs(obj - f) <= rel * (1 + abs(f))


def test_share_qp_and_update_costs():
    p = W.rt_qp(n=600, seed=31)
    a = ipm.Solver(tol_kkt=1e-8).set_qp_rt(p)
    b = ipm.Solver(tol_kkt=1e-8).share_qp(a)
    ba, bb = a.device_bytes(), b.device_bytes()
    assert ba["matrix_refs"] == 2 and bb["matrix"] == ba["matrix"] and bb["state"] == ba["state"]
    a.solve_async()
    b.solve_async()
    assert a.wait() == ipm.IPM_OK and b.wait() == ipm.IPM_OK
    xa = a.get()["x"]
    assert np.array_equal(xa, b.get()["x"])
    # new costs on b only: same result as a fresh handle loaded with them
    w2, c2, _ = W.request_costs(p, dict(seed=5))
    b.update_costs(f_w=w2, c=c2)
    assert b.solve() == ipm.IPM_OK
    xb = b.get()["x"]
    p2 = _rt_with(p, w2, c2)
    with ipm.Solver(tol_kkt=1e-8) as f:
        f.set_qp_rt(p2)
        assert f.solve() == ipm.IPM_OK
        assert np.array_equal(xb, f.get()["x"])
    assert a.solve() == ipm.IPM_OK and np.array_equal(a.get()["x"], xa)
    # the matrices outlive the handle that loaded them
    a.close()
    assert b.device_bytes()["matrix_refs"] == 1
    assert b.solve() == ipm.IPM_OK
    out = b.get()
    assert np.array_equal(out["x"], xb)
    assert kkt_check.rel_kkt(kkt_check.rt_ops(p2), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-8
    assert _obj_close(p2, out["info"]["primal_obj"])
    b.close()


def test_share_qp_rejects_bad_pairs():
    p = W.rt_qp(n=200, seed=32)
    a = ipm.Solver().set_qp_rt(p)
    with pytest.raises(ipm.IpmError) as e:
        ipm.Solver(storage="bf16").share_qp(a)
    assert e.value.status == ipm.IPM_ERR_ARG
    with pytest.raises(ipm.IpmError) as e:
        ipm.Solver().share_qp(ipm.Solver())
    assert e.value.status == ipm.IPM_ERR_STATE
    a.close()


def test_warm_chain_converges_faster_and_matches_oracle():
    p = W.rt_qp(n=1500, seed=33)
    req = dict(seed=77)
    with ipm.Solver(tol_kkt=1e-6, storage="bf16") as s:
        s.set_qp_rt(p)
        prev, iters = None, []
        for k in range(4):
            prev = W.request_costs(p, req, prev)
            s.update_costs(f_w=prev[0], c=prev[1])
            assert s.solve(warm=k > 0) == ipm.IPM_OK
            out = s.get()
            iters.append(out["info"]["ipm_iters"])
        assert max(iters[1:]) < iters[0]
        pk = _rt_with(p, prev[0], prev[1])
        assert kkt_check.rel_kkt(kkt_check.rt_ops(pk), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-6
        assert _obj_close(pk, out["info"]["primal_obj"])


@pytest.mark.parametrize("storage", ["bf16", "f64"])
def test_serving_mix_equals_alone(storage):
    plans = W.rt_batch(count=5, seed=3, scale=0.03)
    reqs = W.serving_stream(horizon=0.3, lam=60.0, chain_frac=0.4, chain_len=3, n_plans=5, seed=4)
    assert any(r["steps"] == 3 for r in reqs) and any(r["steps"] == 1 for r in reqs)
    opts = dict(tol_kkt=1e-6, storage=storage)
    srv = serve.Server(plans, budget_bytes=1e12, max_inflight=4, keep_x=True, **opts)
    srv.budget = srv.used + 2 * max(srv.state_bytes)      # forces waits and slot reuse
    qrec, rrec = srv.run(reqs)
    srv.close()
    assert len(qrec) == sum(r["steps"] for r in reqs)
    assert srv.stats["max_inflight_seen"] > 1 and srv.stats["slots_created"] >= 1
    assert all(r["status"] == ipm.IPM_OK and r["rel_kkt"] <= 1e-6 for r in qrec)
    by = {(r["rid"], r["step"]): r for r in qrec}
    for r in reqs:
        plan = plans[r["plan"]]
        with ipm.Solver(**opts) as s:
            s.set_qp_rt(plan)
            prev = None
            for k in range(r["steps"]):
                prev = W.request_costs(plan, r, prev)
                s.update_costs(f_w=prev[0], c=prev[1])
                assert s.solve(warm=k > 0) == ipm.IPM_OK
                out = s.get()
                rec = by[(r["rid"], k)]
                assert np.array_equal(out["x"], rec["x"]), (r["rid"], k)
                assert out["info"]["ipm_iters"] == rec["ipm_iters"]
    # the last QP of every chain against the independent checker
    for r in reqs:
        if r["steps"] > 1:
            prev = None
            for k in range(r["steps"]):
                prev = W.request_costs(plans[r["plan"]], r, prev)
            pk = _rt_with(plans[r["plan"]], prev[0], prev[1])
            x = by[(r["rid"], r["steps"] - 1)]["x"]
            qp = O.from_rt(pk)
            ref, info = O.solve(qp, tol=1e-10)
            assert info.status == "optimal"
            assert abs(O.objective(qp, x) - O.objective(qp, ref.x)) <= 1e-6 * (1 + abs(O.objective(qp, ref.x)))


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_concurrent_slots_bitwise_equal(storage):
    """Many solves in flight at once on their own streams: slots of one RT plan (low-rank
    stiff-row correction factored on the device) and of a dense plan (the DENSE
    preconditioner), three rounds.  Contention delays some blocks of every launch past others
    of the same launch, so a kernel whose blocks read what another block of it writes gives
    different results here; every solve must equal the solve alone, bitwise."""
    import torch
    rt = W.rt_qp(n=6000, seed=41)
    dn = W.dense_qp(n=400, m=800, seed=42)
    opts = dict(tol_kkt=1e-6, storage=storage)

    def load(kind, s):
        if kind == "rt":
            s.set_qp_rt(rt)
        else:
            s.set_qp_dense(dn["H"], dn["c"], dn["A"], dn["b"], dn["l"], dn["u"])
        return s

    ref = {}
    for kind in ("rt", "dense") if storage == "f64" else ("rt",):
        with load(kind, ipm.Solver(**opts)) as s:
            assert s.solve() == ipm.IPM_OK
            out = s.get()
            ref[kind] = (out["x"].copy(), out["info"]["ipm_iters"], out["info"]["cg_iters"])
    plans = {k: load(k, ipm.Solver(**opts)) for k in ref}
    slots = []
    for kind in ref:
        for _ in range(6 if kind == "rt" else 4):
            st = torch.cuda.Stream()
            slots.append((kind, ipm.Solver(**opts).share_qp(plans[kind], stream=st.cuda_stream), st))
    if "rt" in ref:
        stiff = plans["rt"]
        stiff.solve()
        assert stiff.get()["info"]["max_stiff_rows"] > 32    # the stiff factor spans several tiles
    for _ in range(3):
        for kind, s, st in slots:
            s.solve_async(stream=st.cuda_stream)
        for kind, s, st in slots:
            assert s.wait() == ipm.IPM_OK
            out = s.get(stream=st.cuda_stream)
            x, it, cg = ref[kind]
            assert out["info"]["ipm_iters"] == it and out["info"]["cg_iters"] == cg, (kind, out["info"])
            assert np.array_equal(out["x"], x), kind
    for _, s, _ in slots:
        s.close()
    for s in plans.values():
        s.close()
