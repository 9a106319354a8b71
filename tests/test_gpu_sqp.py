"""SQP outer loop with its QP sub-problems on the GPU (quasi-Newton Hessian updated through
ipm_set_lowrank, costs through ipm_update_costs, warm starts) against the same loop with
the oracle's sub-problem solves."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2405_03584_gb300 import ipm, sqp, workloads as W

pytestmark = pytest.mark.gpu


def _objective(p):
    D = sp.csr_matrix((p["D_data"], p["D_indices"], p["D_indptr"]), shape=(p["V"], p["n"]))
    obj = sqp.DoseObjective(D, p["target"], p["presc"], p["organ"], p["soft_max"], p["w_target"], p["w_organ"])
    return obj, D[p["a_rows"]]


def test_sqp_gpu_matches_oracle_subproblems():
    from tests.test_sqp_host import OracleQP
    p = W.sqp_problem(n=400, density=0.02, seed=8)
    obj, A = _objective(p)
    with ipm.Solver(tol_kkt=1e-9, precond="jacobi_lr", u_cap=120) as s:
        res = sqp.sqp_solve(obj, A, p["b"], p["l"], p["u"], np.zeros(p["n"]), s, max_iter=150, tol=1e-6, u_cap=120)
    assert res.converged, res.history[-1]
    assert all(h["qp_status"] == ipm.IPM_OK for h in res.history)
    obj2, _ = _objective(p)
    ref = sqp.sqp_solve(obj2, A, p["b"], p["l"], p["u"], np.zeros(p["n"]), OracleQP(), max_iter=150, tol=1e-6,
                        u_cap=120)
    assert ref.converged
    assert abs(res.f - ref.f) <= 1e-6 * (1 + abs(ref.f))
    assert np.abs(res.x - ref.x).max() <= 1e-3 * (1 + np.abs(ref.x).max())
    cold = res.history[0]["qp_ipm_iters"]
    warm = np.mean([h["qp_ipm_iters"] for h in res.history[1:]])
    assert warm < cold


def test_sqp_gpu_two_sided_rows():
    """The SQP loop with two-sided rows (dose windows beside the hard organ limits, the
    paper's l_A <= A x <= u_A): GPU sub-problems against the oracle's, signed multipliers."""
    from tests.test_sqp_host import OracleQP, two_sided_rows
    p = W.sqp_problem(n=120, density=0.05, seed=5)
    obj, A = _objective(p)
    A2, b2, bl2, xf = two_sided_rows(p, obj, A, 5, 12)
    with ipm.Solver(tol_kkt=1e-9, precond="jacobi_lr", u_cap=120) as s:
        res = sqp.sqp_solve(obj, A2, b2, p["l"], p["u"], xf, s, max_iter=150, tol=1e-6, u_cap=120, bl=bl2)
    assert res.converged, res.history[-1]
    assert all(h["qp_status"] == ipm.IPM_OK for h in res.history)
    obj2, _ = _objective(p)
    ref = sqp.sqp_solve(obj2, A2, b2, p["l"], p["u"], xf, OracleQP(), max_iter=150, tol=1e-6, u_cap=120, bl=bl2)
    assert ref.converged
    assert abs(res.f - ref.f) <= 1e-6 * (1 + abs(ref.f))
    assert np.abs(res.x - ref.x).max() <= 1e-3 * (1 + np.abs(ref.x).max())
    big = np.abs(ref.y) > 1e-3 * np.abs(ref.y).max()
    assert (ref.y[big] < 0).any() and np.all(np.sign(res.y[big]) == np.sign(ref.y[big]))


def test_set_lowrank_capacity_and_reset():
    p = W.bfgs_qp(n=300, k=6, seed=31)
    with ipm.Solver(tol_kkt=1e-8, u_cap=16) as s:
        s.set_qp_bfgs(p)
        assert s.solve() == ipm.IPM_OK
        x_full = s.get()["x"]
        with pytest.raises(ipm.IpmError) as e:
            s.set_lowrank(np.zeros((p["n"], 17)), np.zeros(17))
        assert e.value.status == ipm.IPM_ERR_TOO_LARGE
        # dropping the term and putting it back reproduces the first solve
        s.set_lowrank(None, None)
        assert s.solve() == ipm.IPM_OK
        x_h0 = s.get()["x"]
        assert np.abs(x_h0 - x_full).max() > 1e-6
        s.set_lowrank(p["U"], p["uw"])
        assert s.solve() == ipm.IPM_OK
        assert np.array_equal(s.get()["x"], x_full)
