"""Independent certificate checker: relative KKT residual of any primal-dual point.

Test infrastructure only (see the package docstring).  It shares no code with the CUDA
library and none with ``oracle.ipm`` either: it evaluates every product with its own
sparse matrix-vector routines, so it can grade points at the full RT sizes where no dense
matrix fits.

Problem: min 0.5 x^T H x + c^T x  s.t.  A x <= b,  l <= x <= u  (Section 3.1 eq:qp with the
bounds separated, Section 4).  The relative KKT residual (the paper defines none; this is
the reading used for every parity claim) is the maximum of

  primal : max(||max(A x - b, 0)||_inf, ||max(l - x, 0)||_inf, ||max(x - u, 0)||_inf) / (1 + ||b||_inf)
  dual   : ||H x + c + A^T y - z_l + z_u||_inf / (1 + max(||c||_inf, ||H x||_inf, ||A^T y||_inf))
  gap    : |pobj - dobj| / (1 + |pobj| + |dobj|)

with pobj = 0.5 x^T H x + c^T x and the Lagrangian dual value
dobj = -0.5 x^T H x - b^T y + l^T z_l - u^T z_u (y, z clipped at 0; z_l (z_u) counted only
where l (u) is finite).

Two-sided rows bl <= A x <= b (the paper's l_A <= A x <= u_A; either side may be infinite)
carry one signed multiplier y per row: y_u = max(y, 0) belongs to the upper side, y_l =
max(-y, 0) to the lower side, each counted only where its side is finite.  Then A^T y above
is A^T (y_u - y_l), the primal part also measures max(bl - A x, 0), ||b||_inf runs over both
sides' finite values and dobj has -b^T y_u + bl^T y_l in place of -b^T y.
"""
from __future__ import annotations

import numpy as np

__all__ = ["Operators", "dense_ops", "rt_ops", "bfgs_ops", "rel_kkt", "rt_condensed_entries", "rt_residual_dual"]


class Operators:
    """H x, A x and A^T y for one QP, plus its vectors."""

    def __init__(self, Hx, Ax, Aty, c, b, l, u, bl=None):
        self.Hx, self.Ax, self.Aty = Hx, Ax, Aty
        self.c, self.b, self.l, self.u = (np.asarray(v, float) for v in (c, b, l, u))
        self.bl = None if bl is None else np.asarray(bl, float)


def _csr_mv(indptr, indices, data, x, nrows):
    """y = M x for a CSR matrix, by a segmented sum of data * x[indices]."""
    rows = np.repeat(np.arange(nrows), np.diff(indptr))
    return np.bincount(rows, weights=data * x[indices], minlength=nrows)


def _csr_tmv(indptr, indices, data, y, ncols):
    """x = M^T y for a CSR matrix, by a scatter of data * y[row] into the columns."""
    nz = np.diff(indptr)
    rows = np.repeat(np.arange(nz.shape[0]), nz)
    return np.bincount(indices, weights=data * y[rows], minlength=ncols)


def dense_ops(p: dict) -> Operators:
    H, A = np.asarray(p["H"], float), np.asarray(p["A"], float).reshape(-1, len(p["c"]))
    return Operators(lambda x: H @ x, lambda x: A @ x, lambda y: A.T @ y, p["c"], p["b"], p["l"], p["u"],
                     p.get("bl"))


def rt_ops(p: dict) -> Operators:
    """Operators of an RT-shaped QP: H x = D^T (w o (D x)) + h0 o x, A = D[a_rows]."""
    ip, ix, dv = p["D_indptr"], p["D_indices"], p["D_data"]
    V, n = p["V"], p["n"]
    w, h0 = np.asarray(p["w"], float), np.asarray(p["h0"], float)
    ar = np.asarray(p["a_rows"], dtype=np.int64)

    def Hx(x):
        return _csr_tmv(ip, ix, dv, w * _csr_mv(ip, ix, dv, x, V), n) + h0 * x

    def Ax(x):
        return _csr_mv(ip, ix, dv, x, V)[ar]

    def Aty(y):
        full = np.zeros(V)
        np.add.at(full, ar, y)
        return _csr_tmv(ip, ix, dv, full, n)

    return Operators(Hx, Ax, Aty, p["c"], p["b"], p["l"], p["u"], p.get("bl"))


def bfgs_ops(p: dict) -> Operators:
    """Operators of a QP with a quasi-Newton Hessian: H x = h0 o x + U (w o (U^T x)), A in CSR."""
    U, w, h0 = np.asarray(p["U"], float), np.asarray(p["uw"], float), np.asarray(p["h0"], float)
    n, m = p["n"], p["m"]

    def Hx(x):
        return h0 * x + U @ (w * (U.T @ x))

    if m:
        ip, ix, dv = p["A_indptr"], p["A_indices"], p["A_data"]
        Ax = lambda x: _csr_mv(ip, ix, dv, x, m)
        Aty = lambda y: _csr_tmv(ip, ix, dv, y, n)
    else:
        Ax = lambda x: np.zeros(0)
        Aty = lambda y: np.zeros(n)
    return Operators(Hx, Ax, Aty, p["c"], p["b"], p["l"], p["u"])


def rel_kkt(ops: Operators, x, y, zl, zu, detail: bool = False):
    """Relative KKT residual (max of the primal, dual and gap parts, see module docstring)."""
    x = np.asarray(x, float)
    y = np.asarray(y, float)
    if ops.bl is None:                       # one-sided rows A x <= b
        fb, fbl = np.ones(y.shape[0], bool), np.zeros(y.shape[0], bool)
    else:
        fb, fbl = np.isfinite(ops.b), np.isfinite(ops.bl)
    bu = np.where(fb, ops.b, 0.0)
    bl = np.where(fbl, ops.bl, 0.0) if ops.bl is not None else np.zeros(y.shape[0])
    yu = np.where(fb, np.maximum(y, 0.0), 0.0)
    yl = np.where(fbl, np.maximum(-y, 0.0), 0.0)
    fl, fu = np.isfinite(ops.l), np.isfinite(ops.u)
    zl = np.where(fl, np.maximum(np.asarray(zl, float), 0.0), 0.0)
    zu = np.where(fu, np.maximum(np.asarray(zu, float), 0.0), 0.0)
    Hx, Ax, Aty = ops.Hx(x), ops.Ax(x), ops.Aty(yu - yl)
    nb = max(np.max(np.abs(bu), initial=0.0), np.max(np.abs(bl), initial=0.0))
    viol = max(np.max(np.where(fb, np.maximum(Ax - bu, 0.0), 0.0), initial=0.0),
               np.max(np.where(fbl, np.maximum(bl - Ax, 0.0), 0.0), initial=0.0),
               np.max(np.where(fl, np.maximum(np.where(fl, ops.l, 0.0) - x, 0.0), 0.0), initial=0.0),
               np.max(np.where(fu, np.maximum(x - np.where(fu, ops.u, 0.0), 0.0), 0.0), initial=0.0))
    primal = viol / (1.0 + nb)
    rd = Hx + ops.c + Aty - zl + zu
    dual = np.max(np.abs(rd), initial=0.0) / (1.0 + max(np.max(np.abs(ops.c), initial=0.0),
                                                         np.max(np.abs(Hx), initial=0.0),
                                                         np.max(np.abs(Aty), initial=0.0)))
    pobj = 0.5 * x @ Hx + ops.c @ x
    dobj = -0.5 * x @ Hx - bu @ yu + bl @ yl + np.sum(np.where(fl, np.where(fl, ops.l, 0.0) * zl, 0.0)) \
        - np.sum(np.where(fu, np.where(fu, ops.u, 0.0) * zu, 0.0))
    gap = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    val = float(max(primal, dual, gap))
    if detail:
        return val, dict(primal=float(primal), dual=float(dual), gap=float(gap), pobj=float(pobj), dobj=float(dobj))
    return val


def rt_residual_dual(p: dict, x, y, zl, zu):
    """r_d = H x + c + A^T y - z_l + z_u for an RT-shaped QP (eq:perturbed_KKT's r_H)."""
    ops = rt_ops(p)
    fl, fu = np.isfinite(ops.l), np.isfinite(ops.u)
    return ops.Hx(x) + ops.c + ops.Aty(y) - np.where(fl, zl, 0.0) + np.where(fu, zu, 0.0)


def rt_condensed_entries(p: dict, x, s, y, zl, zu, pvec, cols):
    """Selected entries q_j, j in cols, of q = (H + A^T Theta A + Sigma) p for an RT-shaped QP,
    each evaluated on its own from the definition (no full matrix product):

        q_j = sum_{i : D_ij != 0} D_ij (w_i + theta~_i) (D_i . p) + (h0_j + sigma_j) p_j,

    theta~_i = y_k / s_k when voxel row i is constraint k (a_rows[k] = i), else 0;
    sigma_j = z_l,j / (x_j - l_j) + z_u,j / (u_j - x_j) over the finite bounds.
    Used at full problem sizes, where only sampled entries are affordable on the host."""
    ip, ix, dv = p["D_indptr"], p["D_indices"], p["D_data"]
    V = p["V"]
    theta_row = np.zeros(V)
    theta_row[np.asarray(p["a_rows"], dtype=np.int64)] = np.asarray(y, float) / np.asarray(s, float)
    l, u = np.asarray(p["l"], float), np.asarray(p["u"], float)
    out = np.empty(len(cols))
    for t, j in enumerate(cols):
        acc = 0.0
        # rows whose column list holds j: scan by binary search in each row's sorted columns
        for i in _rows_with_col(ip, ix, j):
            seg = slice(ip[i], ip[i + 1])
            dij = dv[seg][np.searchsorted(ix[seg], j)]
            acc += dij * (p["w"][i] + theta_row[i]) * (dv[seg] @ pvec[ix[seg]])
        sig = 0.0
        if np.isfinite(l[j]):
            sig += zl[j] / (x[j] - l[j])
        if np.isfinite(u[j]):
            sig += zu[j] / (u[j] - x[j])
        out[t] = acc + (p["h0"][j] + sig) * pvec[j]
    return out


_COL_CACHE = {}


def _rows_with_col(ip, ix, j):
    """Row indices i with column j present (cached column index of the matrix)."""
    key = (id(ip), id(ix))
    if key not in _COL_CACHE:
        _COL_CACHE.clear()
        rows = np.repeat(np.arange(ip.shape[0] - 1), np.diff(ip))
        order = np.argsort(ix, kind="stable")
        cnt = np.bincount(ix, minlength=int(ix.max()) + 1 if ix.size else 1)
        ptr = np.concatenate([[0], np.cumsum(cnt)])
        _COL_CACHE[key] = (rows[order], ptr)
    rws, ptr = _COL_CACHE[key]
    return rws[ptr[j]:ptr[j + 1]]
