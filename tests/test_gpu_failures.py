"""Every failure status of the C ABI, reached on purpose in forms that cannot hang or fault
the GPU: iteration limits, a PCG that cannot meet its tolerance, a device-memory budget
below what the QP needs, a host wall-clock limit shorter than the solve, and a batch whose
member changed after the batch was captured.  In each case the library reports the status,
the handle stays usable, and a following normal call succeeds."""
import time

import numpy as np
import pytest

from oracle import kkt_check
from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_03584_gb300 import build
    build.build()
    ipm.load()


def test_max_iter():
    p = W.rt_qp(n=600, seed=81)
    with ipm.Solver(tol_kkt=1e-8, max_ipm=1) as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_MAX_ITER
        assert s.get()["info"]["ipm_iters"] == 1
    with ipm.Solver(tol_kkt=1e-8) as s:      # the same QP with the default limit converges
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK


@pytest.mark.parametrize("storage,refine_mode", [("f64", 0), ("bf16", 0), ("bf16", 1)])
def test_cg_stall(storage, refine_mode):
    """One PCG iteration per Newton step against a tolerance of 1e-12: the first direction
    (residual far above 1e-2 of its right-hand side) is tolerated, the second ends the solve
    with IPM_CG_STALL."""
    p = W.rt_qp(n=1200, seed=82)
    with ipm.Solver(tol_kkt=1e-8, max_cg=1, cg_eta_min=1e-12, cg_eta_max=1e-12, storage=storage, refine_max=1,
                    refine_mode=refine_mode) as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_CG_STALL
        info = s.get()["info"]
        assert info["ipm_iters"] == 2, info
        assert all(t["pcg_converged"] == 0 and t["pcg_rel_residual"] > 1e-2 for t in s.trace())
        # the iterate is kept and stays strictly interior
        out = s.get()
        assert np.all(out["x"] > p["l"]) and np.all(out["x"] < p["u"]) and np.all(out["s"] > 0)


def test_memory_budget():
    p = W.rt_qp(n=600, seed=83)
    with ipm.Solver(mem_budget=1e5) as s:
        with pytest.raises(ipm.IpmError) as e:
            s.set_qp_rt(p)
        assert e.value.status == ipm.IPM_ERR_OOM
        with pytest.raises(ipm.IpmError) as e:
            s.solve()
        assert e.value.status == ipm.IPM_ERR_STATE
    with ipm.Solver() as plan, ipm.Solver(mem_budget=1e5) as slot:
        plan.set_qp_rt(p)
        with pytest.raises(ipm.IpmError) as e:
            slot.share_qp(plan)                  # even the per-handle state exceeds the budget
        assert e.value.status == ipm.IPM_ERR_OOM
        need = plan.device_bytes()
        with ipm.Solver(mem_budget=float(need["state"] + (1 << 20))) as ok:
            ok.share_qp(plan)
            assert ok.solve() == ipm.IPM_OK


def test_host_timeout_then_collect():
    """timeout_ms shorter than the solve: ipm_solve returns IPM_ERR_TIMEOUT while the solve
    keeps running on the device; other calls on the handle are refused until it is collected,
    then the collected result is the converged one."""
    p = W.rt_qp(n=8000, seed=84)
    with ipm.Solver(tol_kkt=1e-7, timeout_ms=0.2) as s:
        s.set_qp_rt(p)
        with pytest.raises(ipm.IpmError) as e:
            s.solve()
        assert e.value.status == ipm.IPM_ERR_TIMEOUT
        with pytest.raises(ipm.IpmError) as e:
            s.get()
        assert e.value.status == ipm.IPM_ERR_STATE
        t0 = time.time()
        while not s.done():
            assert time.time() - t0 < 120, "solve did not finish"
            time.sleep(0.01)
        assert s.wait() == ipm.IPM_OK
        out = s.get()
        assert kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-7
    # the asynchronous form: ipm_solve_wait itself runs out of time, a later wait collects
    with ipm.Solver(tol_kkt=1e-7, timeout_ms=0.2) as s:
        s.set_qp_rt(p)
        s.solve_async()
        with pytest.raises(ipm.IpmError) as e:
            s.wait()
        assert e.value.status == ipm.IPM_ERR_TIMEOUT
        t0 = time.time()
        while not s.done():
            assert time.time() - t0 < 120
            time.sleep(0.01)
        assert s.wait() == ipm.IPM_OK


@pytest.mark.parametrize("storage,arith", [("f64", "df32"), ("bf16", "f64")])
def test_device_wait_limit(storage, arith):
    """The staged rows pass waits on mbarriers for its bulk copies; every wait is bounded.
    wait_test arms the first tile's barrier for 16 bytes more than is copied, so that wait
    runs out (after wait_limit_ms) with every copy landed: the block records the timeout and
    stops the PCG loop, the solve ends with IPM_ERR_TIMEOUT after its first IPM iteration, and
    the GPU context stays usable for the next solve."""
    p = W.rt_qp(n=4000, seed=85)
    opts = dict(tol_kkt=1e-7, storage=storage, op_arith=arith, rows_format="runs", rows_stage=1)
    with ipm.Solver(wait_test=1, wait_limit_ms=5.0, **opts) as s:
        s.set_qp_rt(p)
        with pytest.raises(ipm.IpmError) as e:
            s.solve()
        assert e.value.status == ipm.IPM_ERR_TIMEOUT
        assert s.info()["ipm_iters"] == 1
    with ipm.Solver(**opts) as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK
        out = s.get()
        assert kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-7


def test_batch_refuses_changed_member():
    """A batch captures each member's buffers; after ipm_set_qp, ipm_share_qp or
    ipm_set_lowrank on a member, ipm_batch_solve refuses to launch (IPM_ERR_STATE)."""
    probs = [W.rt_qp(n=n, seed=90 + n) for n in (300, 410)]
    solvers = []
    for q in probs:
        s = ipm.Solver(tol_kkt=1e-8)
        s.set_qp_rt(q)
        solvers.append(s)
    b = ipm.Batch(solvers)
    assert b.solve() == [ipm.IPM_OK, ipm.IPM_OK]
    x0 = solvers[0].get()["x"]
    solvers[0].set_qp_rt(probs[0])           # reload: the captured buffers are gone
    with pytest.raises(ipm.IpmError) as e:
        b.solve()
    assert e.value.status == ipm.IPM_ERR_STATE
    b.close()
    b = ipm.Batch(solvers)                   # a new capture works, with the same result
    assert b.solve() == [ipm.IPM_OK, ipm.IPM_OK]
    assert np.array_equal(solvers[0].get()["x"], x0)
    b.close()
    plan = solvers[1]
    slot = ipm.Solver(tol_kkt=1e-8)
    slot.share_qp(plan)
    b = ipm.Batch([solvers[0], slot])
    assert b.solve() == [ipm.IPM_OK, ipm.IPM_OK]
    slot.share_qp(plan)                      # a new state arena for the slot
    with pytest.raises(ipm.IpmError) as e:
        b.solve()
    assert e.value.status == ipm.IPM_ERR_STATE
    b.close()
    slot.close()
    # the low-rank Hessian term: its column count is baked into the captured kernels
    q = W.bfgs_qp(n=500, k=3, seed=5)
    with ipm.Solver(tol_kkt=1e-8, u_cap=8) as s:
        s.set_qp_bfgs(q)
        b = ipm.Batch([s])
        assert b.solve() == [ipm.IPM_OK]
        s.set_lowrank(q["U"][:, :4], q["uw"][:4])
        with pytest.raises(ipm.IpmError) as e:
            b.solve()
        assert e.value.status == ipm.IPM_ERR_STATE
        b.close()
    for s in solvers:
        s.close()
