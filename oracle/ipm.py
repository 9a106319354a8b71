"""Plain CPU FP64 primal-dual interior point method with dense Cholesky Newton steps.

Test infrastructure only: used by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py``.  It shares no code with the CUDA library.

Problem (the paper's QP, Section 3.1 eq:qp, with a one-sided constraint block and the
variable bounds separated as in Section 4 before eq:2x2_reduced):

    min 0.5 x^T H x + c^T x   s.t.   A x + s = b,  s >= 0,   l <= x <= u.

Unknowns: x (n), slack s (m), multipliers y (m) for A x <= b, z_l (n) for x >= l and
z_u (n) for x <= u (zero where that bound is infinite).  The bound slacks are implicit:
t_l = x - l, t_u = u - x.

Everything here is dense numpy; a library routine (Cholesky, triangular solve) serves as a
single step.  Each function names the passage it follows.  Readings of points the paper
leaves open (the sign of the upper-row residual, the norm in the mu test, the start point,
tau, the stop rule) are stated where they are used.

Two-sided rows l_A <= A x <= u_A (the paper's form before eq:2x2_reduced) enter through
``two_sided``: the stack B = [A; -A] turns them into the one-sided rows above.

Parity pins: the closed form x = -H^{-1} c (unconstrained), per-coordinate clipping
(separable box QP, also with two-sided single-variable rows), brute-force active-set
enumeration (n <= 8; three states per two-sided row), the full unreduced Newton system
(eq:newton_system), the doubly augmented system (eq:2x2_augmented) and the complementarity /
duality-gap identities; see tests/test_oracle_pins.py.

Parity unpinned: the iteration path.  The start point, the norm of the mu test, and with
them the step-length sequence and the iteration counts follow readings of points the paper
leaves open; the pins fix those readings' invariants (a strictly interior start, a norm
that vanishes exactly on the central path) and the results the path reaches, not the path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

__all__ = [
    "DenseQP", "Iterate", "from_dense", "from_rt", "residuals", "scaled_residual_norm",
    "condensed_system", "newton_direction", "doubly_augmented_direction", "step_lengths",
    "start_point", "solve", "objective", "complementarity_mean", "two_sided", "row_multipliers",
]


@dataclass
class DenseQP:
    H: np.ndarray          # n x n, symmetric positive definite
    c: np.ndarray          # n
    A: np.ndarray          # m x n
    b: np.ndarray          # m
    l: np.ndarray          # n, may hold -inf
    u: np.ndarray          # n, may hold +inf

    @property
    def n(self):
        return self.c.shape[0]

    @property
    def m(self):
        return self.b.shape[0]

    @property
    def fl(self):
        return np.isfinite(self.l)

    @property
    def fu(self):
        return np.isfinite(self.u)


@dataclass
class Iterate:
    x: np.ndarray
    s: np.ndarray
    y: np.ndarray
    zl: np.ndarray
    zu: np.ndarray

    def copy(self):
        return Iterate(self.x.copy(), self.s.copy(), self.y.copy(), self.zl.copy(), self.zu.copy())


def from_dense(p: dict) -> DenseQP:
    return DenseQP(np.asarray(p["H"], float), np.asarray(p["c"], float), np.asarray(p["A"], float).reshape(-1, p["c"].shape[0]),
                   np.asarray(p["b"], float), np.asarray(p["l"], float), np.asarray(p["u"], float))


def from_rt(p: dict) -> DenseQP:
    """Dense form of an RT-shaped QP: H = D^T diag(w) D + diag(h0), A = D[a_rows]."""
    n, V = p["n"], p["V"]
    D = np.zeros((V, n))
    rows = np.repeat(np.arange(V), np.diff(p["D_indptr"]))
    D[rows, p["D_indices"]] = p["D_data"]
    H = D.T @ (p["w"][:, None] * D) + np.diag(p["h0"])
    H = 0.5 * (H + H.T)
    A = D[np.asarray(p["a_rows"], dtype=np.int64)]
    return DenseQP(H, np.asarray(p["c"], float), A, np.asarray(p["b"], float),
                   np.asarray(p["l"], float), np.asarray(p["u"], float))


def from_bfgs(p: dict) -> DenseQP:
    """Dense form of a QP with a quasi-Newton Hessian (Section 3.3, eq:bfgs_hessian):
    H = diag(h0) + U diag(w) U^T; A from its CSR arrays (or none)."""
    n, m = p["n"], p["m"]
    U, w = np.asarray(p["U"], float), np.asarray(p["uw"], float)
    H = np.diag(np.asarray(p["h0"], float)) + (U * w) @ U.T
    H = 0.5 * (H + H.T)
    A = np.zeros((m, n))
    if m:
        rows = np.repeat(np.arange(m), np.diff(p["A_indptr"]))
        A[rows, p["A_indices"]] = p["A_data"]
    return DenseQP(H, np.asarray(p["c"], float), A, np.asarray(p["b"], float),
                   np.asarray(p["l"], float), np.asarray(p["u"], float))


def two_sided(H, c, A, bl, bu, l, u):
    """One-sided form of two-sided rows bl <= A x <= bu (Section 4, before eq:2x2_reduced:
    B = [A; -A] with the upper and lower row bounds).  Rows whose upper side is +inf drop out
    of the first block, rows whose lower side is -inf out of the second.  Returns
    (DenseQP, upper, lower): the original indices of the rows in each block."""
    A = np.asarray(A, float)
    bl, bu = np.asarray(bl, float), np.asarray(bu, float)
    upper = np.flatnonzero(np.isfinite(bu))
    lower = np.flatnonzero(np.isfinite(bl))
    B = np.vstack([A[upper], -A[lower]]).reshape(-1, A.shape[1])
    b = np.concatenate([bu[upper], -bl[lower]])
    return DenseQP(np.asarray(H, float), np.asarray(c, float), B, b, np.asarray(l, float),
                   np.asarray(u, float)), upper, lower


def row_multipliers(y, upper, lower, m):
    """Multiplier of each original two-sided row from the stacked ones: the upper row's minus
    the lower row's (the row's own sign convention: > 0 at its upper side, < 0 at its lower)."""
    out = np.zeros(m)
    np.add.at(out, upper, y[:upper.shape[0]])
    np.add.at(out, lower, -y[upper.shape[0]:])
    return out


def _tl(qp, x):
    return np.where(qp.fl, x - np.where(qp.fl, qp.l, 0.0), 1.0)


def _tu(qp, x):
    return np.where(qp.fu, np.where(qp.fu, qp.u, 0.0) - x, 1.0)


def residuals(qp: DenseQP, it: Iterate, mu: float):
    """Perturbed KKT residuals (Section 3.1, eq:perturbed_KKT) for A x <= b and the box.

    r_d = H x + c + A^T y - z_l + z_u      (the paper's r_H with lambda_u -> y, bound rows split)
    r_p = A x + s - b                      (reading: the upper-row residual is A x + s - b with
                                            s >= 0; the paper prints three different signs)
    r_s = s o y - mu,  r_l = t_l o z_l - mu,  r_u = t_u o z_u - mu   (r_c1, r_c2)
    r_l / r_u are zero where the bound is infinite.
    """
    tl, tu = _tl(qp, it.x), _tu(qp, it.x)
    rd = qp.H @ it.x + qp.c + qp.A.T @ it.y - it.zl + it.zu
    rp = qp.A @ it.x + it.s - qp.b
    rs = it.s * it.y - mu
    rl = np.where(qp.fl, tl * it.zl - mu, 0.0)
    ru = np.where(qp.fu, tu * it.zu - mu, 0.0)
    return rd, rp, rs, rl, ru


def complementarity_mean(qp: DenseQP, it: Iterate) -> float:
    """Average complementarity product over the m rows and the finite bounds."""
    tl, tu = _tl(qp, it.x), _tu(qp, it.x)
    tot = it.s @ it.y + np.sum(np.where(qp.fl, tl * it.zl, 0.0)) + np.sum(np.where(qp.fu, tu * it.zu, 0.0))
    cnt = qp.m + int(qp.fl.sum()) + int(qp.fu.sum())
    return float(tot / max(cnt, 1))


def scaled_residual_norm(qp: DenseQP, it: Iterate, res) -> float:
    """The ||r|| of Algorithm 1's mu test (reading; the paper leaves the norm open).

        ||r|| = max( ||(r_s, r_l, r_u)||_inf,  (1 + |f(x)|) / N_c * max(e_p, e_d) )

    with e_p = ||r_p||_inf / (1 + ||b||_inf), e_d = ||r_d||_inf / (1 + ||c||_inf), f the
    objective and N_c the number of complementarity pairs (m plus the finite bounds).
    The complementarity part is absolute (units of mu).  The primal and dual parts are
    relative; (1 + |f|) / N_c turns them into the same units, so that "||r|| < mu" asks for
    relative infeasibility no larger than the relative duality gap N_c mu / (1 + |f|) of
    the central point for mu.
    """
    rd, rp, rs, rl, ru = res
    ep = np.max(np.abs(rp), initial=0.0) / (1.0 + np.max(np.abs(qp.b), initial=0.0))
    ed = np.max(np.abs(rd), initial=0.0) / (1.0 + np.max(np.abs(qp.c), initial=0.0))
    ec = max(np.max(np.abs(rs), initial=0.0), np.max(np.abs(rl), initial=0.0), np.max(np.abs(ru), initial=0.0))
    nc = max(1, qp.m + int(qp.fl.sum()) + int(qp.fu.sum()))
    return float(max(ec, (1.0 + abs(objective(qp, it.x))) / nc * max(ep, ed)))


def condensed_system(qp: DenseQP, it: Iterate, res):
    """Normal-equations form of the Newton system (Section 4, eq:2x2_reduced with B = -A,
    D = Theta^{-1}, after eliminating the constraint multipliers).

    Eliminating dz_l, dz_u, ds and dy from eq:newton_system gives
        (H + A^T Theta A + Sigma) dx = -r_d - r_l / t_l + r_u / t_u - A^T (theta o r_p - r_s / s)
    with theta = y / s and Sigma = diag(z_l / t_l + z_u / t_u) (zero terms at infinite bounds).
    Returns (K, rhs, theta, sigma).
    """
    rd, rp, rs, rl, ru = res
    tl, tu = _tl(qp, it.x), _tu(qp, it.x)
    theta = it.y / it.s
    sigma = np.where(qp.fl, it.zl / tl, 0.0) + np.where(qp.fu, it.zu / tu, 0.0)
    K = qp.H + qp.A.T @ (theta[:, None] * qp.A) + np.diag(sigma)
    rhs = -rd - np.where(qp.fl, rl / tl, 0.0) + np.where(qp.fu, ru / tu, 0.0) - qp.A.T @ (theta * rp - rs / it.s)
    return K, rhs, theta, sigma


def recover_direction(qp: DenseQP, it: Iterate, res, dx):
    """Back-substitution for (ds, dy, dz_l, dz_u) from dx (Algorithm 1's recovery of
    the full direction): the last four block rows of eq:newton_system solved for them."""
    rd, rp, rs, rl, ru = res
    tl, tu = _tl(qp, it.x), _tu(qp, it.x)
    Adx = qp.A @ dx
    ds = -rp - Adx
    dy = (it.y / it.s) * (Adx + rp) - rs / it.s
    dzl = np.where(qp.fl, (-rl - it.zl * dx) / tl, 0.0)
    dzu = np.where(qp.fu, (-ru + it.zu * dx) / tu, 0.0)
    return Iterate(dx, ds, dy, dzl, dzu)


def newton_direction(qp: DenseQP, it: Iterate, mu: float):
    """Exact Newton direction of eq:newton_system: dense Cholesky on the condensed system,
    then back-substitution."""
    res = residuals(qp, it, mu)
    K, rhs, _, _ = condensed_system(qp, it, res)
    dx = sla.cho_solve(sla.cho_factor(K, lower=True), rhs)
    return recover_direction(qp, it, res, dx)


def doubly_augmented_direction(qp: DenseQP, it: Iterate, mu: float):
    """The paper's own symmetric positive definite form (Section 4, eq:2x2_augmented):

        [[Q + 2 B^T D^{-1} B, B^T], [B, D]] [dx; dl] = [r1 + 2 B^T D^{-1} r2; r2]

    with Q = H + Sigma, B = -A, D = Theta^{-1} = diag(s / y), r1 = -r_d - r_l/t_l + r_u/t_u
    and r2 = r_p - r_s / y (eq:2x2_reduced's right-hand side for this sign convention).
    Solved densely; used to cross-check the condensed direction.  Returns (dx, dy).
    """
    rd, rp, rs, rl, ru = residuals(qp, it, mu)
    tl, tu = _tl(qp, it.x), _tu(qp, it.x)
    sigma = np.where(qp.fl, it.zl / tl, 0.0) + np.where(qp.fu, it.zu / tu, 0.0)
    Q = qp.H + np.diag(sigma)
    B = -qp.A
    Dd = it.s / it.y
    r1 = -rd - np.where(qp.fl, rl / tl, 0.0) + np.where(qp.fu, ru / tu, 0.0)
    r2 = rp - rs / it.y
    n, m = qp.n, qp.m
    K = np.zeros((n + m, n + m))
    K[:n, :n] = Q + 2.0 * B.T @ (B / Dd[:, None])
    K[:n, n:] = B.T
    K[n:, :n] = B
    K[n:, n:] = np.diag(Dd)
    rhs = np.concatenate([r1 + 2.0 * B.T @ (r2 / Dd), r2])
    sol = sla.cho_solve(sla.cho_factor(K, lower=True), rhs)
    return sol[:n], sol[n:]


def _max_ratio(v, dv, mask=None):
    """Largest a with v + a dv >= 0 over the entries with dv < 0 (inf if none)."""
    neg = dv < 0
    if mask is not None:
        neg = neg & mask
    if not np.any(neg):
        return np.inf
    return float(np.min(-v[neg] / dv[neg]))


def step_lengths(qp: DenseQP, it: Iterate, d: Iterate, tau: float = 0.995, equal: bool = False):
    """Fraction-to-boundary step lengths (Section 3.1 line search; Algorithm 1's
    separate primal and dual step lengths).

    alpha_p = min(1, tau * max{a : s + a ds >= 0, t_l + a dx >= 0, t_u - a dx >= 0})
    alpha_d = min(1, tau * max{a : y + a dy >= 0, z_l + a dz_l >= 0, z_u + a dz_u >= 0})
    tau = 0.995 (reading: the paper states no fraction).  ``equal`` takes min(alpha_p, alpha_d)
    for both.
    """
    tl, tu = _tl(qp, it.x), _tu(qp, it.x)
    ap = min(_max_ratio(it.s, d.s), _max_ratio(tl, d.x, qp.fl), _max_ratio(tu, -d.x, qp.fu))
    ad = min(_max_ratio(it.y, d.y), _max_ratio(it.zl, d.zl, qp.fl), _max_ratio(it.zu, d.zu, qp.fu))
    ap = min(1.0, tau * ap)
    ad = min(1.0, tau * ad)
    if equal:
        ap = ad = min(ap, ad)
    return ap, ad


def start_point(qp: DenseQP):
    """Initial point (reading; the paper only notes that any positive slack is a valid
    start, Section 3.1 after the slack reformulation).

    x0  = 0 projected into the box shrunk by delta_j = 0.1 min(1, (u_j - l_j) / 2)
          (delta_j = 0.1 for a one-sided bound; x0_j = 0 for a free variable);
    s0  = max(b - A x0, 1);
    with g = H x0 + c:  z_l0 = max(1, g), z_u0 = max(1, -g) on finite bounds (0 elsewhere),
    y0  = 1 on every row (so that theta = y / s starts moderate and no constraint row begins
          "stiff");
    mu0 = the average complementarity product of this point.
    Returns (Iterate, mu0).
    """
    n = qp.n
    both = qp.fl & qp.fu
    width = np.where(both, np.where(qp.fu, qp.u, 0.0) - np.where(qp.fl, qp.l, 0.0), 2.0)
    delta = 0.1 * np.minimum(1.0, 0.5 * width)
    lo = np.where(qp.fl, np.where(qp.fl, qp.l, 0.0) + delta, -np.inf)
    hi = np.where(qp.fu, np.where(qp.fu, qp.u, 0.0) - delta, np.inf)
    x0 = np.clip(np.zeros(n), lo, hi)
    s0 = np.maximum(qp.b - qp.A @ x0, 1.0)
    g = qp.H @ x0 + qp.c
    zl0 = np.where(qp.fl, np.maximum(1.0, g), 0.0)
    zu0 = np.where(qp.fu, np.maximum(1.0, -g), 0.0)
    y0 = np.ones(qp.m)
    it = Iterate(x0, s0, y0, zl0, zu0)
    return it, complementarity_mean(qp, it)


def objective(qp: DenseQP, x):
    return float(0.5 * x @ (qp.H @ x) + qp.c @ x)


@dataclass
class SolveInfo:
    status: str = "max_iter"
    iterations: int = 0
    mu: float = 0.0
    rel_kkt: float = np.inf
    history: list = field(default_factory=list)


def _rel_kkt_inline(qp: DenseQP, it: Iterate):
    """Relative KKT residual used only for the oracle's own stop rule (the independent
    checker in kkt_check.py is what tests grade with)."""
    Hx = qp.H @ it.x
    Aty = qp.A.T @ it.y
    rd = Hx + qp.c + Aty - it.zl + it.zu
    ep = np.max(np.maximum(qp.A @ it.x - qp.b, 0.0), initial=0.0) / (1.0 + np.max(np.abs(qp.b), initial=0.0))
    ed = np.max(np.abs(rd), initial=0.0) / (1.0 + max(np.max(np.abs(qp.c), initial=0.0), np.max(np.abs(Hx), initial=0.0), np.max(np.abs(Aty), initial=0.0)))
    pobj = 0.5 * it.x @ Hx + qp.c @ it.x
    dobj = -0.5 * it.x @ Hx - qp.b @ it.y + np.sum(np.where(qp.fl, qp.l, 0.0) * it.zl) - np.sum(np.where(qp.fu, qp.u, 0.0) * it.zu)
    eg = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    return float(max(ep, ed, eg))


def solve(qp: DenseQP, tol: float = 1e-8, tau: float = 0.995, max_iter: int = 200,
          equal_steps: bool = False, mu_floor_rel: float = 1e-16, record: bool = False):
    """Algorithm 1 with exact Newton steps.

    Per iteration: Newton direction (dense Cholesky on the condensed system), step lengths
    alpha_p (x, s) and alpha_d (y, z), update, residuals, then the mu test:
    if ||r|| < mu (scaled_residual_norm): mu <- mu / 10.
    Stop rule (reading of "if mu <= mu_tol return"): return once the relative KKT residual
    of the iterate is <= tol.  Returns (Iterate, SolveInfo).
    """
    it, mu0 = start_point(qp)
    mu = mu0
    info = SolveInfo()
    if record:
        info.history.append(dict(k=-1, mu=mu, ap=0.0, ad=0.0, rn=np.nan, rel_kkt=_rel_kkt_inline(qp, it), obj=objective(qp, it.x)))
    for k in range(max_iter):
        d = newton_direction(qp, it, mu)
        ap, ad = step_lengths(qp, it, d, tau, equal_steps)
        it.x = it.x + ap * d.x
        it.s = it.s + ap * d.s
        it.y = it.y + ad * d.y
        it.zl = it.zl + ad * d.zl
        it.zu = it.zu + ad * d.zu
        res = residuals(qp, it, mu)
        rk = _rel_kkt_inline(qp, it)
        rn = scaled_residual_norm(qp, it, res)
        if record:
            tl, tu = _tl(qp, it.x), _tu(qp, it.x)
            pos = min(np.min(it.s, initial=np.inf), np.min(it.y, initial=np.inf),
                      np.min(np.where(qp.fl, tl, np.inf), initial=np.inf), np.min(np.where(qp.fu, tu, np.inf), initial=np.inf),
                      np.min(np.where(qp.fl, it.zl, np.inf), initial=np.inf), np.min(np.where(qp.fu, it.zu, np.inf), initial=np.inf))
            info.history.append(dict(k=k, mu=mu, ap=ap, ad=ad, rn=rn, rel_kkt=rk, obj=objective(qp, it.x), min_pos=float(pos)))
        info.iterations = k + 1
        info.rel_kkt = rk
        if rk <= tol:
            info.status = "optimal"
            break
        if rn < mu:
            mu = max(mu / 10.0, mu_floor_rel * mu0)
    info.mu = mu
    return it, info
