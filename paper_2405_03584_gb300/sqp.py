"""SQP outer loop around the GPU IPM (Sections 3.2 and 3.3).

The paper's solver sits inside an SQP method: every SQP iteration solves one convex QP
sub-problem whose Hessian is a BFGS approximation kept in compact form (eq:bfgs_hessian,
H = H0 + U W U^T, two columns per iteration), warm-started from the previous sub-problem.
This module is that outer loop for a smooth objective with linear constraints; the
objective stands in for the planning system's dose objectives (not available) and all of
its arithmetic is host-side (numpy / scipy): the QP sub-problems are the library's.

Sub-problem of iteration k, in the variables x themselves (so the constraints and bounds
never change and the previous solution is a valid warm start):

    min 0.5 x^T H_k x + (g_k - H_k x_k)^T x   s.t.   A x <= b,  l <= x <= u,

whose solution x* gives the step d = x* - x_k; x_{k+1} = x_k + alpha d with a backtracking
(Armijo) line search on f (the feasible set is convex, so every alpha in [0, 1] is feasible).
BFGS update with s = x_{k+1} - x_k, y = g_{k+1} - g_k when y^T s > 0: U gains the columns
H_k s (weight -1 / s^T H_k s) and y (weight 1 / y^T s); when U is full it is dropped
(H = H0 again), as the paper's reset of the quasi-Newton Hessian.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

__all__ = ["DoseObjective", "SQPResult", "sqp_solve"]


class DoseObjective:
    """f(x) = sum_t w_t max(0, p_t - (D x)_t)^2 + sum_o w_o max(0, (D x)_o - m_o)^2 + eps/2 |x|^2

    over target voxels t (prescription p) and organ voxels o (soft limit m): one-sided
    quadratic under- and overdose penalties, continuously differentiable.  D is a scipy CSR
    matrix (voxels x spots)."""

    def __init__(self, D, target, presc, organ, soft_max, w_target, w_organ, eps=1e-4):
        self.D = D.tocsr()
        self.DT = self.D.T.tocsr()
        self.target = np.asarray(target, dtype=np.int64)
        self.organ = np.asarray(organ, dtype=np.int64)
        self.presc = np.asarray(presc, float)
        self.soft_max = np.asarray(soft_max, float)
        self.w_target = np.asarray(w_target, float)
        self.w_organ = np.asarray(w_organ, float)
        self.eps = float(eps)
        self.evals = 0

    def value_grad(self, x):
        self.evals += 1
        dose = self.D @ x
        under = np.maximum(0.0, self.presc - dose[self.target])
        over = np.maximum(0.0, dose[self.organ] - self.soft_max)
        f = float(self.w_target @ under ** 2 + self.w_organ @ over ** 2 + 0.5 * self.eps * (x @ x))
        r = np.zeros(dose.shape[0])
        r[self.target] = -2.0 * self.w_target * under
        r[self.organ] += 2.0 * self.w_organ * over
        return f, self.DT @ r + self.eps * x

    def gauss_newton_diag(self):
        """2 sum_i w_i D_ij^2 over every penalised voxel + eps: the initial Hessian H0."""
        wv = np.zeros(self.D.shape[0])
        wv[self.target] += self.w_target
        wv[self.organ] += self.w_organ
        D2 = self.D.multiply(self.D)
        return 2.0 * (D2.T @ wv) + self.eps


@dataclass
class SQPResult:
    x: np.ndarray
    f: float
    iterations: int
    converged: bool
    history: list = field(default_factory=list)
    y: np.ndarray = None      # multipliers of the last sub-problem (A x <= b, x >= l, x <= u)
    zl: np.ndarray = None
    zu: np.ndarray = None


def _hx(h0, U, w, v):
    out = h0 * v
    if U.shape[1]:
        out = out + U @ (w * (U.T @ v))
    return out


def sqp_solve(obj: DoseObjective, A, b, l, u, x0, solver, max_iter=50, tol=1e-6, u_cap=200, warm=True,
              armijo=1e-4, bl=None):
    """Runs the SQP loop.  ``solver`` is a loaded handle-like object (``ipm.Solver`` with
    ``u_cap`` columns reserved) offering set_qp, update_costs, set_lowrank, solve and get.
    A is a scipy CSR matrix (m x n); bl, if given, makes the rows two-sided (bl <= A x <= b,
    the paper's l_A <= A x <= u_A; b may then hold +inf) and the returned y signed (upper
    side minus lower side).  x0 must be feasible (the line search stays on the segment to
    the sub-problem's solution).  Returns an SQPResult; history has one dict per iteration."""
    n = x0.shape[0]
    x = np.asarray(x0, float).copy()
    h0 = obj.gauss_newton_diag()
    U = np.zeros((n, 0))
    w = np.zeros(0)
    f, g = obj.value_grad(x)
    A = A.tocsr()
    m = A.shape[0]
    two = {} if bl is None else {"bl": np.asarray(bl, float)}
    solver.set_qp(n, m, g - _hx(h0, U, w, x), b if m else None, l, u, h0=h0,
                  A=(A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)) if m else None,
                  **two)
    hist = []
    converged = False
    for k in range(max_iter):
        t0 = time.perf_counter()
        st = solver.solve(warm=warm and k > 0)
        retried = False
        if st != 0 and warm and k > 0:
            # a warm start from the previous solution can stall the interior point method (its
            # complementarity products start far from the central path of the new QP): the
            # sub-problem is solved again from the cold start point before its step is taken
            st = solver.solve(warm=False)
            retried = True
        out = solver.get()
        t_qp = time.perf_counter() - t0
        xs = out["x"]
        d = xs - x
        # optimality of the current point: the sub-problem's step vanishes
        dn = float(np.abs(d).max())
        rec = dict(k=k, f=f, step_inf=dn, qp_status=int(st), qp_ipm_iters=out["info"]["ipm_iters"],
                   qp_cg_iters=out["info"]["cg_iters"], qp_rel_kkt=out["info"]["rel_kkt"], qp_s=t_qp,
                   u_cols=int(U.shape[1]), warm=bool(warm and k > 0), qp_cold_retry=retried)
        if dn <= tol * (1.0 + float(np.abs(x).max())):
            hist.append(rec)
            converged = True
            break
        # backtracking line search on f along d (directional derivative g^T d < 0)
        gd = float(g @ d)
        alpha = 1.0
        while True:
            xn = x + alpha * d
            fn, gn = obj.value_grad(xn)
            if fn <= f + armijo * alpha * gd or alpha < 1e-8:
                break
            alpha *= 0.5
        rec["alpha"] = alpha
        hist.append(rec)
        if fn > f:                                   # no decrease along d: stop where we are
            break
        s = xn - x
        y = gn - g
        sy = float(s @ y)
        if U.shape[1] + 2 > u_cap:
            U, w = np.zeros((n, 0)), np.zeros(0)          # reset to H0
        if sy > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            Hs = _hx(h0, U, w, s)
            U = np.concatenate([U, Hs[:, None], y[:, None]], axis=1)
            w = np.concatenate([w, [-1.0 / float(s @ Hs), 1.0 / sy]])
        x, f, g = xn, fn, gn
        solver.set_lowrank(np.ascontiguousarray(U) if U.shape[1] else None, w if U.shape[1] else None)
        solver.update_costs(c=g - _hx(h0, U, w, x))
    return SQPResult(x=x, f=f, iterations=len(hist), converged=converged, history=hist,
                     y=out["y"], zl=out["zl"], zu=out["zu"])
