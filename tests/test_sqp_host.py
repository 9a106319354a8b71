"""The SQP outer loop (Sections 3.2-3.3) on the CPU: sub-problems solved by the oracle, the
result pinned against scipy's SLSQP on a tiny instance, BFGS compact form and secant
condition along the iterations, monotone objective, stationarity at the end."""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

from oracle import ipm as O
from paper_2405_03584_gb300 import sqp, workloads as W


class OracleQP:
    """Handle-like stand-in for ipm.Solver whose solves are the oracle's (dense, exact steps)."""

    def __init__(self):
        self.U = None
        self.w = None

    def set_qp(self, n, m, c, b=None, l=None, u=None, h0=None, A=None, bl=None, **kw):
        self.n, self.m, self.c, self.b, self.l, self.u, self.h0 = n, m, c, b, l, u, h0
        self.bl = bl
        self.A = np.zeros((m, n))
        if m:
            ip, ix, dv = A
            rows = np.repeat(np.arange(m), np.diff(ip))
            self.A[rows, ix] = dv
        self.U, self.w = np.zeros((n, 0)), np.zeros(0)
        return self

    def set_lowrank(self, U=None, u_w=None):
        self.U = np.zeros((self.n, 0)) if U is None else np.asarray(U)
        self.w = np.zeros(0) if U is None else np.asarray(u_w)

    def update_costs(self, f_w=None, c=None):
        self.c = c

    def solve(self, warm=False):
        H = np.diag(self.h0) + (self.U * self.w) @ self.U.T
        H = 0.5 * (H + H.T)
        if self.bl is None:
            qp = O.DenseQP(H, self.c, self.A, self.b if self.m else np.zeros(0), self.l, self.u)
        else:
            qp, up, lo = O.two_sided(H, self.c, self.A, self.bl, self.b, self.l, self.u)
        self.it, info = O.solve(qp, tol=1e-10)
        if self.bl is not None:
            self.it.y = O.row_multipliers(self.it.y, up, lo, self.m)
        self.info = info
        return 0 if info.status == "optimal" else 3

    def get(self):
        return dict(x=self.it.x, y=self.it.y, zl=self.it.zl, zu=self.it.zu,
                    info=dict(ipm_iters=self.info.iterations, cg_iters=0, rel_kkt=self.info.rel_kkt))


def _objective(p):
    D = sp.csr_matrix((p["D_data"], p["D_indices"], p["D_indptr"]), shape=(p["V"], p["n"]))
    obj = sqp.DoseObjective(D, p["target"], p["presc"], p["organ"], p["soft_max"], p["w_target"], p["w_organ"])
    A = D[p["a_rows"]]
    return obj, A


def test_sqp_matches_slsqp_on_a_tiny_problem():
    p = W.sqp_problem(n=30, density=0.1, seed=3)
    obj, A = _objective(p)
    res = sqp.sqp_solve(obj, A, p["b"], p["l"], p["u"], np.zeros(p["n"]), OracleQP(), max_iter=200, tol=1e-6)
    assert res.converged and res.iterations < 80
    fs = [h["f"] for h in res.history]
    assert all(b <= a + 1e-12 * (1 + abs(a)) for a, b in zip(fs, fs[1:]))
    # independent solution: SLSQP on the same problem
    cons = [{"type": "ineq", "fun": lambda x: p["b"] - A @ x, "jac": lambda x: -A.toarray()}]
    ref = so.minimize(lambda x: obj.value_grad(x), np.zeros(p["n"]), jac=True, method="SLSQP",
                      bounds=list(zip(p["l"], p["u"])), constraints=cons,
                      options=dict(ftol=1e-14, maxiter=2000))
    # (SLSQP may stop on its own precision limit; its value is the comparison)
    assert abs(res.f - ref.fun) <= 1e-7 * (1 + abs(ref.fun))
    # stationarity with the last sub-problem's multipliers: g + A^T y - z_l + z_u = 0
    _, g = obj.value_grad(res.x)
    r = g + A.T @ res.y - res.zl + res.zu
    assert np.abs(r).max() <= 1e-5 * (1 + np.abs(g).max())


def test_sqp_bfgs_secant_and_reset():
    p = W.sqp_problem(n=40, density=0.08, seed=4)
    obj, A = _objective(p)
    rec = {}

    class Spy(OracleQP):
        def set_lowrank(self, U=None, u_w=None):
            super().set_lowrank(U, u_w)
            rec.setdefault("cols", []).append(self.U.shape[1])
            rec["last"] = (self.U.copy(), self.w.copy())

    res = sqp.sqp_solve(obj, A, p["b"], p["l"], p["u"], np.zeros(p["n"]), Spy(), max_iter=12, tol=0.0, u_cap=10)
    cols = rec["cols"]
    assert max(cols) <= 10 and any(c < d for c, d in zip(cols[1:], cols)), cols      # the reset happened
    U, w = rec["last"]
    h0 = obj.gauss_newton_diag()
    H = np.diag(h0) + (U * w) @ U.T
    # the newest pair satisfies the secant condition H s = y; H stays positive definite
    assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() > 0
    s_last, y_last = None, None
    if U.shape[1]:
        y_last = U[:, -1]
        s_last = np.linalg.lstsq(H, y_last, rcond=None)[0]
        np.testing.assert_allclose(H @ s_last, y_last, rtol=1e-8, atol=1e-10)


def test_dose_objective_gradient_and_h0():
    """The objective's gradient against central differences; H0 against the Gauss-Newton
    diagonal written out densely."""
    p = W.sqp_problem(n=25, density=0.2, seed=5)
    obj, _ = _objective(p)
    rng = np.random.default_rng(1)
    x = rng.uniform(0.0, 1.5, size=p["n"])
    f, g = obj.value_grad(x)
    h = 1e-6
    fd = np.array([(obj.value_grad(x + h * e)[0] - obj.value_grad(x - h * e)[0]) / (2 * h) for e in np.eye(p["n"])])
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * (1 + np.abs(g).max()))
    D = obj.D.toarray()
    wv = np.zeros(D.shape[0])
    wv[p["target"]] += p["w_target"]
    wv[p["organ"]] += p["w_organ"]
    np.testing.assert_allclose(obj.gauss_newton_diag(), 2.0 * (D ** 2).T @ wv + obj.eps, rtol=1e-12)


def two_sided_rows(p, obj, A, seed, k):
    """The hard organ rows plus dose windows (0.8, 1.2) x (D x_f) on k non-target voxels,
    the last one lower-only, around x_f = alpha 1 (alpha: half the tightest organ limit),
    which is strictly feasible and serves as the start.  Returns (A, b, bl, x_f)."""
    D = obj.D
    rowsum = np.asarray(abs(D).sum(axis=1)).ravel()
    ar = np.asarray(p["a_rows"])
    xf = np.full(p["n"], 0.5 * np.min(p["b"] / rowsum[ar]))
    taken = np.zeros(p["V"], bool)
    taken[ar] = True
    cand = np.flatnonzero(~taken & (rowsum > 0) & np.isin(np.arange(p["V"]), obj.organ))
    other = np.sort(np.random.default_rng(seed).choice(cand, k, replace=False))
    A2 = sp.vstack([A, D[other]]).tocsr()
    dxf = D[other] @ xf
    b2 = np.concatenate([p["b"], 1.2 * dxf])
    bl2 = np.concatenate([np.full(ar.size, -np.inf), 0.8 * dxf])
    b2[-1] = np.inf
    return A2, b2, bl2, xf


@pytest.mark.parametrize("seed", [5, 6])
def test_sqp_two_sided_rows_match_slsqp(seed):
    """Two-sided rows (the paper's l_A <= A x <= u_A) through the SQP loop: dose windows
    (0.8, 1.2) x (D x_f) on six non-target voxels around the feasible start x_f (one of them
    lower-only) beside the hard organ limits; the result matches SLSQP with both sides as
    inequalities, some lower sides bind, and stationarity holds with the signed multipliers."""
    p = W.sqp_problem(n=30, density=0.1, seed=seed)
    obj, A = _objective(p)
    A2, b2, bl2, xf = two_sided_rows(p, obj, A, seed, 6)
    res = sqp.sqp_solve(obj, A2, b2, p["l"], p["u"], xf, OracleQP(), max_iter=200, tol=1e-6, bl=bl2)
    assert res.converged
    fu, fl = np.isfinite(b2), np.isfinite(bl2)
    cons = [{"type": "ineq", "fun": lambda x: (b2 - A2 @ x)[fu]},
            {"type": "ineq", "fun": lambda x: (A2 @ x - bl2)[fl]}]
    ref = so.minimize(lambda x: obj.value_grad(x), xf, jac=True, method="SLSQP",
                      bounds=list(zip(p["l"], p["u"])), constraints=cons, options=dict(ftol=1e-14, maxiter=2000))
    assert abs(res.f - ref.fun) <= 1e-7 * (1 + abs(ref.fun))
    Ax = A2 @ res.x
    assert np.all(Ax[fu] <= b2[fu] + 1e-7) and np.all(Ax[fl] >= bl2[fl] - 1e-7)
    assert (res.y < -1e-8).any(), "a lower side must bind"
    _, g = obj.value_grad(res.x)
    r = g + A2.T @ res.y - res.zl + res.zu
    assert np.abs(r).max() <= 1e-4 * (1 + np.abs(g).max())


def test_failed_warm_start_is_solved_again_cold():
    """A warm-started sub-problem that ends without converging (a stalled warm start) is solved
    again from the cold start point before its step is taken; the loop then reaches the same
    point as with cold starts throughout."""
    p = W.sqp_problem(n=40, density=0.08, seed=4)
    obj, A = _objective(p)
    calls = []

    class WarmFails(OracleQP):
        def solve(self, warm=False):
            calls.append(warm)
            st = super().solve(warm)
            return 3 if warm else st          # every warm start "stalls" (IPM_MAX_ITER)

    res = sqp.sqp_solve(obj, A, p["b"], p["l"], p["u"], np.zeros(p["n"]), WarmFails(), max_iter=200, tol=1e-6)
    ref = sqp.sqp_solve(obj, A, p["b"], p["l"], p["u"], np.zeros(p["n"]), OracleQP(), max_iter=200, tol=1e-6,
                        warm=False)
    assert res.converged and ref.converged
    assert all(r["qp_status"] == 0 for r in res.history)
    assert all(r["qp_cold_retry"] == (r["k"] > 0) for r in res.history)
    assert calls[0] is False and calls[1:3] == [True, False]
    assert abs(res.f - ref.f) <= 1e-10 * (1 + abs(ref.f))
