"""GPU parity for the quasi-Newton Hessian H = H0 + U W U^T (Section 3.3, eq:bfgs_hessian):
operator, residuals and diagonal against the oracle's dense H, solves of the paper's two
problem shapes (bounds only; many sparse upper and lower constraint rows) at small sizes
against the oracle, and at the paper's full sizes against the independent checker."""
import numpy as np
import pytest

from oracle import ipm as O
from oracle import kkt_check
from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu

SMALL = [
    ("proton_like_613", lambda: W.bfgs_qp(n=613, k=12, seed=21)),
    ("vmat_like_401", lambda: W.bfgs_qp(n=401, k=6, m_ub=523, m_lb=177, density=0.03, seed=22)),
    ("vmat_target_1342", lambda: W.bfgs_qp(n=1342, k=8, m_ub=5287, m_lb=1575, density=0.1, seed=6,
                                           c_mode="target", ub_fac=1.1, lb_fac=0.9)),
]


@pytest.mark.parametrize("name,make", SMALL, ids=[c[0] for c in SMALL])
def test_bfgs_residuals_operator_diag(name, make):
    p = make()
    qp = O.from_bfgs(p)
    s = ipm.Solver(precond="jacobi").set_qp_bfgs(p)
    x, sl, y, zl, zu = W.random_iterate(qp.n, qp.m, qp.l, qp.u, 7, 1.2)
    it = O.Iterate(x, sl, y, zl, zu)
    mu = 0.21
    s.set_iterate(x, sl, y, zl, zu, mu)
    r = s.residuals()
    rd, rp, rs, rl, ru = O.residuals(qp, it, mu)
    np.testing.assert_allclose(r["rd"], rd, rtol=1e-10, atol=1e-11 * (1 + np.abs(rd).max()))
    if qp.m:
        np.testing.assert_allclose(r["rp"], rp, rtol=1e-10, atol=1e-11 * (1 + np.abs(rp).max()))
    val, det = kkt_check.rel_kkt(kkt_check.bfgs_ops(p), x, y, zl, zu, detail=True)
    assert abs(r["dual"] - det["dual"]) <= 1e-10 * (1 + det["dual"])
    assert abs(r["gap"] - det["gap"]) <= 1e-10 * (1 + det["gap"])
    K, _, _, _ = O.condensed_system(qp, it, (rd, rp, rs, rl, ru))
    rng = np.random.default_rng(3)
    for _ in range(2):
        pv = rng.normal(size=qp.n)
        np.testing.assert_allclose(s.apply_kkt(pv), K @ pv, rtol=1e-10,
                                   atol=1e-12 * np.abs(K).max() * np.abs(pv).max() * qp.n)
    np.testing.assert_allclose(s.precond_diag(), np.diag(K), rtol=1e-11)
    s.close()


@pytest.mark.parametrize("precond", ["jacobi_lr", "dense"])
@pytest.mark.parametrize("name,make", SMALL, ids=[c[0] for c in SMALL])
def test_bfgs_solve_vs_oracle(name, make, precond):
    p = make()
    qp = O.from_bfgs(p)
    with ipm.Solver(tol_kkt=1e-8, precond=precond) as s:
        s.set_qp_bfgs(p)
        assert s.solve() == ipm.IPM_OK
        out = s.get()
    rk = kkt_check.rel_kkt(kkt_check.bfgs_ops(p), out["x"], out["y"], out["zl"], out["zu"])
    assert rk <= 1e-8 * 1.0001, rk
    ref, info = O.solve(qp, tol=1e-10)
    assert info.status == "optimal"
    f, f0 = O.objective(qp, out["x"]), O.objective(qp, ref.x)
    assert abs(f - f0) <= 1e-6 * (1 + abs(f0))
    assert np.abs(out["x"] - ref.x).max() <= 1e-4 * (1 + np.abs(ref.x).max())


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_bfgs_reduced_precision_constraints(storage):
    p = SMALL[1][1]()
    qp = O.from_bfgs(p)
    with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr", storage=storage) as s:
        s.set_qp_bfgs(p)
        assert s.solve() == ipm.IPM_OK
        out = s.get()
    assert kkt_check.rel_kkt(kkt_check.bfgs_ops(p), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-8 * 1.0001
    ref, _ = O.solve(qp, tol=1e-10)
    f, f0 = O.objective(qp, out["x"]), O.objective(qp, ref.x)
    assert abs(f - f0) <= 1e-6 * (1 + abs(f0))


def test_bfgs_shared_and_deterministic():
    p = SMALL[0][1]()
    a = ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr").set_qp_bfgs(p)
    b = ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr").share_qp(a)
    assert a.solve() == ipm.IPM_OK and b.solve() == ipm.IPM_OK
    assert np.array_equal(a.get()["x"], b.get()["x"])
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["proton", "vmat"])
def test_bfgs_full_size_certified(case):
    """The paper's problem sizes (Table 1): proton n = 77373 with 2k = 200 update columns and
    bounds only; VMAT n = 13425 with 52867 upper and 15751 lower constraint rows, 2k = 66, an
    objective that pulls towards a plan (a few hundred constraints active at the solution) and
    up to 1024 rows in the low-rank correction."""
    if case == "proton":
        p = W.bfgs_qp(n=77373, k=100, seed=5)
    else:
        p = W.bfgs_qp(n=13425, k=33, m_ub=52867, m_lb=15751, density=0.01, seed=6, c_mode="target",
                      ub_fac=1.1, lb_fac=0.9)
    with ipm.Solver(tol_kkt=1e-6, precond="jacobi_lr", stiff_max=1024) as s:
        s.set_qp_bfgs(p)
        st = s.solve()
        out = s.get()
    assert st == ipm.IPM_OK, out["info"]
    rk = kkt_check.rel_kkt(kkt_check.bfgs_ops(p), out["x"], out["y"], out["zl"], out["zu"])
    assert rk <= 1e-6 * 1.0001, rk
    assert abs(out["info"]["rel_kkt"] - rk) <= 1e-3 * rk + 1e-12
