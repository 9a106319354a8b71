"""Seeded synthetic QP generators shared by the tests, the bench and the oracle checks.

This module only draws inputs: it holds none of the interior point method's arithmetic.
Every problem has the form of the paper's QP (Section 3.1, eq:qp) written with a
one-sided constraint block and separate variable bounds (Section 4, eq:2x2_reduced
separates the bound rows):

    min 0.5 x^T H x + c^T x   s.t.   A x <= b,   l <= x <= u.

Two families are produced.

* ``dense_qp``: a dense QP (H = Q diag(lam) Q^T, dense A).
* ``rt_qp``: a radiation-therapy shaped QP.  The paper's own problems are exported
  from a commercial planning system and are not available, so a dose-like matrix D
  (voxels x beam spots) stands in: each voxel row holds a few contiguous bands of
  spots, with lognormal values.  H = D^T diag(w) D + eps I is kept in factored form,
  c = -D^T diag(w) d_presc, and the linear constraints are a subset of D's rows
  (organ voxels, A = D[a_rows], b = 0.6).

All arrays are numpy, float64 / int32 / int64.  Sparse matrices are CSR triplets
``(indptr int64, indices int32, data float64)`` with sorted, unique column indices
per row.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "dense_qp", "rt_qp", "rt_two_sided", "rt_batch_sizes", "rt_batch", "perturb_chain_step",
    "serving_stream", "request_costs", "bfgs_qp", "sqp_problem", "csr_to_dense", "random_iterate",
]


def dense_qp(n: int = 500, m: int = 1000, seed: int = 0, lam_lo: float = 1e-3,
             lam_hi: float = 1e2, lo: float = 0.0, hi: float = 10.0) -> dict:
    """Dense QP with a known eigen-decomposition of H.

    A ~ N(0, 1/n); H = Q diag(lam) Q^T with Q a sign-fixed random orthogonal matrix and
    lam log-uniform on [lam_lo, lam_hi]; c ~ N(0, 1); lo <= x <= hi;
    b = A 1 + U(0.1, 1) so that x = 1 is strictly feasible.
    The returned dict carries ``Q`` and ``lam`` as well, for closed-form checks.
    """
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, 1.0 / np.sqrt(n), size=(m, n))
    G = rng.normal(size=(n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    lam = 10.0 ** rng.uniform(np.log10(lam_lo), np.log10(lam_hi), size=n)
    H = (Q * lam[None, :]) @ Q.T
    H = 0.5 * (H + H.T)
    c = rng.normal(size=n)
    b = A @ np.ones(n) + rng.uniform(0.1, 1.0, size=m)
    l = np.full(n, lo)
    u = np.full(n, hi)
    return dict(kind="dense", n=n, m=m, H=H, c=c, A=A, b=b, l=l, u=u, Q=Q, lam=lam)


def _band_rows(rng, V, n, density, main_sd_frac=0.02, max_extra=3):
    """Column structure of a banded dose-like matrix, one block of rows at a time.

    Row i holds k_i ~ Binomial(n, density) entries split into 1 + Binomial(max_extra, 0.5)
    contiguous bands.  The first band is centred near i*n/V + N(0, main_sd_frac*n) (voxel
    order follows spatial order); the extra bands are centred uniformly at random.
    Returns (indptr, indices) with sorted unique columns per row.
    """
    k = rng.binomial(n, density, size=V).astype(np.int64)
    k = np.clip(k, 1, n)
    nb = 1 + rng.binomial(max_extra, 0.5, size=V)
    # split k_i into nb_i band lengths (multinomial with equal weights, every band >= 1 where possible)
    lens = np.zeros((V, max_extra + 1), dtype=np.int64)
    u = rng.random((V, max_extra + 1))
    u[np.arange(max_extra + 1)[None, :] >= nb[:, None]] = 0.0
    u /= u.sum(axis=1, keepdims=True)
    lens = np.floor(u * k[:, None]).astype(np.int64)
    rem = k - lens.sum(axis=1)
    lens[np.arange(V), 0] += rem
    centres = np.empty((V, max_extra + 1))
    centres[:, 0] = (np.arange(V) + 0.5) * (n / V) + rng.normal(0.0, main_sd_frac * n, size=V)
    centres[:, 1:] = rng.uniform(0, n, size=(V, max_extra))
    starts = np.rint(centres - lens / 2.0).astype(np.int64)
    starts = np.clip(starts, 0, np.maximum(n - lens, 0))
    # union of each row's bands without a global sort: order the bands of a row by start,
    # clip every band to begin after the previous bands end, then expand the pieces in order
    ends = starts + lens
    ends = np.where(lens > 0, ends, starts)
    order = np.argsort(np.where(lens > 0, starts, n + 1), axis=1, kind="stable")
    st = np.take_along_axis(starts, order, axis=1)
    en = np.take_along_axis(ends, order, axis=1)
    prev_end = np.maximum.accumulate(np.concatenate([np.zeros((V, 1), np.int64), en[:, :-1]], axis=1), axis=1)
    st = np.maximum(st, prev_end)
    ln = np.maximum(en - st, 0)
    nnz_row = ln.sum(axis=1)
    indptr = np.zeros(V + 1, dtype=np.int64)
    np.cumsum(nnz_row, out=indptr[1:])
    flat_len = ln.ravel()
    sel = flat_len > 0
    L = flat_len[sel]
    off = np.arange(L.sum(), dtype=np.int64) - np.repeat(np.cumsum(L) - L, L)
    cidx = (np.repeat(st.ravel()[sel], L) + off).astype(np.int32)
    return indptr, cidx


def rt_qp(n: int = 50_000, V: int | None = None, density: float = 0.005, seed: int = 1,
          target_frac: float = 0.3, n_organ: int | None = None, b_organ: float = 0.6,
          eps: float = 1e-4, lo: float = 0.0, hi: float = 5.0, w_lo: float = 0.1,
          w_hi: float = 10.0) -> dict:
    """Radiation-therapy shaped QP.

    D: V x n dose-like CSR matrix (banded rows, lognormal(0, 1) values); w ~ U(w_lo, w_hi)
    voxel weights; d_presc = 1 on a seeded target_frac of the voxels, else 0;
    H = D^T diag(w) D + eps I (factored: F = D, weights w, diagonal h0 = eps);
    c = -D^T (w * d_presc); A = D[a_rows] with a_rows = n_organ non-target voxels
    (default 20000 when V = 200000, i.e. V/10), b = b_organ; lo <= x <= hi.
    """
    if V is None:
        V = 4 * n
    if n_organ is None:
        n_organ = V // 10
    rng = np.random.default_rng(seed)
    indptr, indices = _band_rows(rng, V, n, density)
    data = rng.lognormal(0.0, 1.0, size=indices.shape[0])
    w = rng.uniform(w_lo, w_hi, size=V)
    perm = rng.permutation(V)
    n_target = int(round(target_frac * V))
    target = np.sort(perm[:n_target])
    d = np.zeros(V)
    d[target] = 1.0
    non_target = np.sort(perm[n_target:])
    a_rows = np.sort(rng.choice(non_target, size=min(n_organ, non_target.size), replace=False)).astype(np.int32)
    # c = -D^T (w * d): a scatter over the stored rows (a problem definition, not solver arithmetic)
    wd = w * d
    rowid = np.repeat(np.arange(V), np.diff(indptr))
    c = -np.bincount(indices, weights=data * wd[rowid], minlength=n)
    m = a_rows.shape[0]
    return dict(kind="rt", n=n, V=V, m=m, D_indptr=indptr, D_indices=indices, D_data=data,
                w=w, d=d, h0=np.full(n, eps), eps=eps, c=c, a_rows=a_rows,
                b=np.full(m, b_organ), l=np.full(n, lo), u=np.full(n, hi))


def rt_two_sided(p: dict, n_window: int | None = None, delta: float = 0.2, lower_only_frac: float = 0.125,
                 seed: int = 5) -> dict:
    """Adds two-sided rows to an RT-shaped QP from ``rt_qp``: the paper's l_A <= A x <= u_A
    (Section 4, before eq:2x2_reduced).  x_f = alpha 1 with alpha = min_k b_k / (2 rowsum_k)
    over the organ rows is strictly feasible; n_window target voxels and as many other
    voxels (none of them organ rows) get the window (1 -/+ delta) (D x_f)_t, where the cost
    pulls target doses up (upper sides bind) and the others down (lower sides bind); a
    fraction lower_only_frac of the window rows keeps only the lower side (b = +inf).  The
    organ rows keep their upper limit only (bl = -inf); the window rows follow them in a_rows."""
    rng = np.random.default_rng(seed)
    V = p["V"]
    rowsum = np.add.reduceat(p["D_data"], p["D_indptr"][:-1]) * (np.diff(p["D_indptr"]) > 0)
    organ = np.asarray(p["a_rows"], dtype=np.int64)
    alpha = 0.5 * float(np.min(p["b"] / np.maximum(rowsum[organ], 1e-300))) if organ.size else 1.0
    dose_f = alpha * rowsum
    taken = np.zeros(V, bool)
    taken[organ] = True
    cand_t = np.flatnonzero((p["d"] > 0) & ~taken & (dose_f > 0))
    cand_o = np.flatnonzero((p["d"] == 0) & ~taken & (dose_f > 0))
    if n_window is None:
        n_window = max(1, cand_t.size // 10)
    win = np.concatenate([rng.choice(cand_t, size=min(n_window, cand_t.size), replace=False),
                          rng.choice(cand_o, size=min(n_window, cand_o.size), replace=False)])
    win = np.sort(win).astype(np.int32)
    lo = (1.0 - delta) * dose_f[win]
    hi = (1.0 + delta) * dose_f[win]
    hi[rng.random(win.size) < lower_only_frac] = np.inf
    m0 = p["m"]
    q = dict(p)
    q["a_rows"] = np.concatenate([organ, win]).astype(np.int32)
    q["m"] = m0 + win.size
    q["b"] = np.concatenate([p["b"], hi])
    q["bl"] = np.concatenate([np.full(m0, -np.inf), lo])
    q["x_feasible"] = np.full(p["n"], alpha)
    return q


def rt_batch_sizes(count: int = 64, seed: int = 3, n_lo: int = 2000, n_hi: int = 40000,
                   dens_lo: float = 0.002, dens_hi: float = 0.01):
    """Per-instance (n, density, child seed) of the uneven batch: n ~ U[n_lo, n_hi],
    density ~ U[dens_lo, dens_hi]; V = 4n and n/2 constraint rows are implied."""
    ss = np.random.SeedSequence(seed)
    kids = ss.spawn(count)
    rng = np.random.default_rng(ss.spawn(1)[0])
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    dens = rng.uniform(dens_lo, dens_hi, size=count)
    return [(int(ns[i]), float(dens[i]), kids[i]) for i in range(count)]


def rt_batch(count: int = 64, seed: int = 3, scale: float = 1.0, **kw):
    """Uneven batch of RT-shaped QPs (optionally with every n scaled down by ``scale``)."""
    out = []
    for n, dens, kid in rt_batch_sizes(count, seed, **kw):
        nn = max(16, int(round(n * scale)))
        out.append(rt_qp(n=nn, V=4 * nn, density=dens, seed=kid, n_organ=nn // 2))
    return out


def perturb_chain_step(qp: dict, rng: np.random.Generator, rel: float = 0.01) -> dict:
    """Next QP of an SQP-like chain: w <- w (1 + rel xi), c <- c (1 + rel xi), xi ~ N(0, 1).

    w stays positive for rel * |xi| < 1, so H = D^T W D + eps I stays positive definite.
    """
    q = dict(qp)
    q["w"] = qp["w"] * (1.0 + rel * rng.normal(size=qp["w"].shape))
    q["w"] = np.maximum(q["w"], 1e-6)
    q["c"] = qp["c"] * (1.0 + rel * rng.normal(size=qp["c"].shape))
    return q


def serving_stream(horizon: float = 60.0, lam: float = 20.0, chain_frac: float = 0.3, chain_len: int = 20,
                   n_plans: int = 64, seed: int = 4) -> list[dict]:
    """Request stream of the serving workload: Poisson arrivals of rate ``lam`` over
    ``horizon`` seconds; each request names a plan (uniform over ``n_plans``) and is a single
    QP or, with probability ``chain_frac``, an SQP-like chain of ``chain_len`` related QPs.
    Each request carries its own seed for the cost perturbations of its QPs."""
    rng = np.random.default_rng(seed)
    out, t, rid = [], 0.0, 0
    while True:
        t += rng.exponential(1.0 / lam)
        if t >= horizon:
            break
        steps = chain_len if rng.random() < chain_frac else 1
        out.append(dict(rid=rid, t=t, plan=int(rng.integers(n_plans)), steps=steps,
                        seed=int(rng.integers(2**62))))
        rid += 1
    return out


def request_costs(plan: dict, req: dict, prev: tuple | None = None, rel: float = 0.01) -> tuple:
    """(f_w, c) of a request's next QP: the first from the plan's own, each later one from
    the previous QP of the chain, by ``perturb_chain_step`` with a generator keyed by the
    request's seed and the step, so any step can be regenerated alone."""
    step = 0 if prev is None else prev[2] + 1
    base = dict(w=plan["w"], c=plan["c"]) if prev is None else dict(w=prev[0], c=prev[1])
    q = perturb_chain_step(base, np.random.default_rng([req["seed"], step]), rel)
    return q["w"], q["c"], step


def bfgs_qp(n: int = 77_373, k: int = 100, m_ub: int = 0, m_lb: int = 0, density: float = 0.01,
            seed: int = 5, lam_lo: float = 1e-2, lam_hi: float = 1e2, c_mode: str = "random",
            ub_fac: float = 1.2, lb_fac: float = 0.8) -> dict:
    """QP sub-problem with a quasi-Newton Hessian in compact form (Section 3.3, eq:bfgs_hessian):
    H = H0 + U diag(w) U^T, H0 = diag(h0), U n x 2k.

    H0 = diag(U(0.5, 2)).  k BFGS updates H <- H - (H s)(H s)^T / (s^T H s) + y y^T / (y^T s)
    from seeded pairs: s ~ N(0, 1/n), y = B s with B = diag(lam), lam log-uniform on
    [lam_lo, lam_hi] (so y^T s > 0 and every H stays positive definite).  Each update appends
    the columns H s (weight -1 / (s^T H s)) and y (weight 1 / (y^T s)) to U; H s is applied
    through the compact form built so far.  c ~ N(0, 1) (c_mode "random"), or c = -H x_t +
    0.1 N(0, 1) with x_t ~ U(0.5, 1.5) (c_mode "target": the objective pulls towards a plan
    x_t); x >= 0 (one bound per variable, no upper bound).  Constraints (m = m_ub + m_lb rows
    of a banded dose-like matrix G with lognormal values, as in ``rt_qp``): upper rows
    G_i x <= ub_fac G_i 1, lower rows written as -G_i x <= -lb_fac G_i 1, so x = 1 is strictly
    feasible.  A is returned as CSR.
    Sizes of the paper's cases (Table 1): proton n = 77373, m = 0 (k up to 100 before spot
    filtering); VMAT n = 13425, m = 52867 upper + 15751 lower rows (k up to 33).  The update
    steps S (n x k) and lam are returned too (y_i = lam o s_i)."""
    rng = np.random.default_rng(seed)
    h0 = rng.uniform(0.5, 2.0, size=n)
    lam = 10.0 ** rng.uniform(np.log10(lam_lo), np.log10(lam_hi), size=n)
    U = np.zeros((n, 2 * k))
    w = np.zeros(2 * k)
    S = np.zeros((n, k))
    for i in range(k):
        sv = rng.normal(0.0, 1.0 / np.sqrt(n), size=n)
        S[:, i] = sv
        yv = lam * sv
        Hs = h0 * sv + U[:, :2 * i] @ (w[:2 * i] * (U[:, :2 * i].T @ sv))
        U[:, 2 * i] = Hs
        w[2 * i] = -1.0 / float(sv @ Hs)
        U[:, 2 * i + 1] = yv
        w[2 * i + 1] = 1.0 / float(yv @ sv)
    c = rng.normal(size=n)
    if c_mode == "target":
        xt = rng.uniform(0.5, 1.5, size=n)
        c = -(h0 * xt + U @ (w * (U.T @ xt))) + 0.1 * c
    m = m_ub + m_lb
    out = dict(kind="bfgs", n=n, m=m, k=k, h0=h0, U=U, uw=w, c=c, l=np.zeros(n), u=np.full(n, np.inf),
               b=np.zeros(m), S=S, lam=lam)
    if m:
        indptr, indices = _band_rows(rng, m, n, density)
        data = rng.lognormal(0.0, 1.0, size=indices.shape[0])
        rowid = np.repeat(np.arange(m), np.diff(indptr))
        g1 = np.bincount(rowid, weights=data, minlength=m)      # G_i . 1
        sign = np.ones(m)
        sign[m_ub:] = -1.0
        out["A_indptr"], out["A_indices"], out["A_data"] = indptr, indices, data * sign[rowid]
        out["b"] = np.where(sign > 0, ub_fac * g1, -lb_fac * g1)
    return out


def sqp_problem(n: int = 5000, density: float = 0.005, seed: int = 7, presc: float = 1.0,
                soft_max: float = 0.5, hard_max: float = 0.8, organ_weight: float = 0.1,
                n_hard: int | None = None) -> dict:
    """Nonlinear planning problem for the SQP driver, built on the RT generator's dose matrix
    (``rt_qp`` with the same n, density and seed): one-sided quadratic penalties, underdose
    below ``presc`` on the target voxels (weights w) and overdose above ``soft_max`` on every
    other voxel (weights organ_weight * w); hard limits A x <= hard_max on n_hard organ rows
    (default n / 20; A = D[a_rows] as in ``rt_qp``); 0 <= x <= 5."""
    p = rt_qp(n=n, density=density, seed=seed, b_organ=hard_max, n_organ=n // 20 if n_hard is None else n_hard)
    V = p["V"]
    target = np.flatnonzero(p["d"] > 0)
    organ = np.flatnonzero(p["d"] == 0)
    return dict(kind="sqp", n=n, V=V, D_indptr=p["D_indptr"], D_indices=p["D_indices"], D_data=p["D_data"],
                target=target, presc=np.full(target.size, presc), w_target=p["w"][target],
                organ=organ, soft_max=np.full(organ.size, soft_max), w_organ=organ_weight * p["w"][organ],
                a_rows=p["a_rows"], b=p["b"], l=p["l"], u=p["u"])


def csr_to_dense(indptr, indices, data, shape):
    """Plain CSR -> dense expansion (test helper)."""
    M = np.zeros(shape)
    rows = np.repeat(np.arange(shape[0]), np.diff(indptr))
    np.add.at(M, (rows, indices), data)
    return M


def random_iterate(n: int, m: int, l: np.ndarray, u: np.ndarray, seed: int, spread: float = 1.0):
    """A strictly interior primal-dual point (x, s, y, z_l, z_u) for operator/direction tests.

    x lies strictly between finite bounds; s, y, z are log-normally spread positive numbers
    (``spread`` sets the log-std, mimicking the widening of y/s late in a solve); z_l (z_u)
    is zero where l (u) is infinite.
    """
    rng = np.random.default_rng(seed)
    lo = np.where(np.isfinite(l), l, -10.0)
    hi = np.where(np.isfinite(u), u, 10.0)
    x = lo + (hi - lo) * rng.uniform(0.05, 0.95, size=n)
    s = np.exp(rng.normal(0, spread, size=m))
    y = np.exp(rng.normal(0, spread, size=m))
    zl = np.where(np.isfinite(l), np.exp(rng.normal(0, spread, size=n)), 0.0)
    zu = np.where(np.isfinite(u), np.exp(rng.normal(0, spread, size=n)), 0.0)
    return x, s, y, zl, zu
