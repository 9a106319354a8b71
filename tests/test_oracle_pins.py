"""Pins for the CPU oracle: each test checks it against something other than itself
(closed forms, hand-solved fixtures, brute force, the paper's unreduced and doubly augmented
Newton systems, exact identities), chosen so that a dropped term, a flipped sign or a
transposed operand in oracle/ipm.py or oracle/kkt_check.py fails at least one of them."""
import json
import os

import numpy as np
import pytest

from oracle import ipm, kkt_check
from paper_2405_03584_gb300 import workloads as W
from tests._bruteforce import solve_bruteforce, solve_bruteforce_two_sided

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tiny_qps.json")


def _rand_qp(n, m, seed, cond=1e2, free_frac=0.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = 10 ** rng.uniform(0, np.log10(cond), size=n)
    H = (Q * lam) @ Q.T
    H = 0.5 * (H + H.T)
    c = rng.normal(size=n) * 3
    A = rng.normal(size=(m, n))
    xf = rng.uniform(-0.5, 0.5, size=n)
    b = A @ xf + rng.uniform(0.05, 1.0, size=m)
    l = rng.uniform(-2, -0.6, size=n)
    u = rng.uniform(0.6, 2, size=n)
    free = rng.random(n) < free_frac
    l[free & (rng.random(n) < 0.5)] = -np.inf
    u[free & (rng.random(n) < 0.5)] = np.inf
    return dict(H=H, c=c, A=A.reshape(m, n), b=b, l=l, u=u)


def _qp_from_json(case):
    n = len(case["c"])
    A = np.array(case["A"], float).reshape(-1, n)
    l = np.array([-np.inf if v is None else v for v in case["l"]], float)
    u = np.array([np.inf if v is None else v for v in case["u"]], float)
    return dict(H=np.array(case["H"], float), c=np.array(case["c"], float), A=A,
                b=np.array(case["b"], float).reshape(-1), l=l, u=u)


# ---------------------------------------------------------------- closed forms

def test_unconstrained_closed_form():
    """No rows, no bounds: the IPM must return x = -H^{-1} c, written here through the
    generator's own eigen-decomposition H = Q diag(lam) Q^T (not through a solver)."""
    p = W.dense_qp(n=60, m=0, seed=11)
    p["A"] = np.zeros((0, 60))
    p["b"] = np.zeros(0)
    p["l"] = np.full(60, -np.inf)
    p["u"] = np.full(60, np.inf)
    x_star = -(p["Q"] @ ((p["Q"].T @ p["c"]) / p["lam"]))
    it, info = ipm.solve(ipm.from_dense(p), tol=1e-12)
    assert info.status == "optimal"
    np.testing.assert_allclose(it.x, x_star, rtol=1e-9, atol=1e-9 * np.abs(x_star).max())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_separable_box_clipping(seed):
    """Diagonal H, no rows: x_j = clip(-c_j / h_j, l_j, u_j) coordinate by coordinate."""
    rng = np.random.default_rng(100 + seed)
    n = 40
    h = 10 ** rng.uniform(-2, 2, size=n)
    c = rng.normal(size=n) * 5
    l = rng.uniform(-3, 0, size=n)
    u = rng.uniform(0.1, 3, size=n)
    l[rng.random(n) < 0.2] = -np.inf
    u[rng.random(n) < 0.2] = np.inf
    p = dict(H=np.diag(h), c=c, A=np.zeros((0, n)), b=np.zeros(0), l=l, u=u)
    it, info = ipm.solve(ipm.from_dense(p), tol=1e-12)
    assert info.status == "optimal"
    np.testing.assert_allclose(it.x, np.clip(-c / h, l, u), rtol=1e-8, atol=1e-9)


def test_hand_solved_fixtures():
    """tests/golden/tiny_qps.json: KKT points derived by hand from eq:perturbed_KKT at mu = 0."""
    cases = json.load(open(GOLD))["cases"]
    for case in cases:
        p = _qp_from_json(case)
        it, info = ipm.solve(ipm.from_dense(p), tol=1e-12)
        assert info.status == "optimal", case["name"]
        np.testing.assert_allclose(it.x, case["x"], atol=1e-8, err_msg=case["name"])
        np.testing.assert_allclose(it.y, case["y"], atol=1e-7, err_msg=case["name"])
        fl, fu = np.isfinite(p["l"]), np.isfinite(p["u"])
        np.testing.assert_allclose(np.where(fl, it.zl, 0), case["zl"], atol=1e-7, err_msg=case["name"])
        np.testing.assert_allclose(np.where(fu, it.zu, 0), case["zu"], atol=1e-7, err_msg=case["name"])
        assert abs(ipm.objective(ipm.from_dense(p), it.x) - case["obj"]) < 1e-9
        # the stored multipliers certify the stored point with the independent checker
        ops = kkt_check.dense_ops(p)
        assert kkt_check.rel_kkt(ops, case["x"], case["y"], case["zl"], case["zu"]) < 1e-14


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n,m,seed", [(2, 1, 0), (3, 2, 1), (4, 3, 2), (5, 3, 3), (6, 4, 4), (6, 2, 5), (8, 2, 6)])
def test_bruteforce_active_set(n, m, seed):
    """Enumerate all 3^n 2^m active sets; the oracle's x must match the enumerated optimum,
    and the enumerated KKT point must certify as optimal in the independent checker."""
    p = _rand_qp(n, m, seed, free_frac=0.2)
    bf = solve_bruteforce(p["H"], p["c"], p["A"], p["b"], p["l"], p["u"])
    assert bf is not None
    f, xb, yb, zlb, zub = bf
    it, info = ipm.solve(ipm.from_dense(p), tol=1e-12)
    assert info.status == "optimal"
    np.testing.assert_allclose(it.x, xb, atol=1e-8)
    assert abs(ipm.objective(ipm.from_dense(p), it.x) - f) <= 1e-9 * (1 + abs(f))
    ops = kkt_check.dense_ops(p)
    assert kkt_check.rel_kkt(ops, xb, yb, zlb, zub) < 1e-12
    assert kkt_check.rel_kkt(ops, it.x, it.y, it.zl, it.zu) < 1e-11


# ---------------------------------------------------------------- Newton systems

def _interior_point(p, seed, spread=1.0):
    n, m = len(p["c"]), len(p["b"])
    return ipm.Iterate(*W.random_iterate(n, m, p["l"], p["u"], seed, spread))


@pytest.mark.parametrize("seed", [0, 1])
def test_newton_direction_solves_unreduced_system(seed):
    """The condensed-Cholesky direction must satisfy the full, unreduced Newton system of
    eq:newton_system (restated for A x + s = b and the separated bounds), assembled here
    block by block in (dx, dy, dz_l, dz_u, ds) order."""
    p = _rand_qp(12, 7, 20 + seed, cond=1e3, free_frac=0.3)
    qp = ipm.from_dense(p)
    it = _interior_point(p, seed, spread=2.0)
    mu = 0.37
    d = ipm.newton_direction(qp, it, mu)
    rd, rp, rs, rl, ru = ipm.residuals(qp, it, mu)
    n, m = qp.n, qp.m
    fl, fu = qp.fl, qp.fu
    tl = np.where(fl, it.x - np.where(fl, qp.l, 0), 1.0)
    tu = np.where(fu, np.where(fu, qp.u, 0) - it.x, 1.0)
    N = 3 * n + 2 * m
    K = np.zeros((N, N))
    ix, iy, izl, izu, isl = 0, n, n + m, 2 * n + m, 3 * n + m
    K[ix:iy, ix:iy] = qp.H
    K[ix:iy, iy:izl] = qp.A.T
    K[ix:iy, izl:izu] = -np.eye(n)
    K[ix:iy, izu:isl] = np.eye(n)
    K[iy:izl, ix:iy] = qp.A                         # A dx + ds = -r_p
    K[iy:izl, isl:] = np.eye(m)
    K[izl:izu, ix:iy] = np.diag(np.where(fl, it.zl, 0))   # z_l dx + t_l dz_l = -r_l
    K[izl:izu, izl:izu] = np.diag(np.where(fl, tl, 1.0))
    K[izu:isl, ix:iy] = -np.diag(np.where(fu, it.zu, 0))  # -z_u dx + t_u dz_u = -r_u
    K[izu:isl, izu:isl] = np.diag(np.where(fu, tu, 1.0))
    K[isl:, iy:izl] = np.diag(it.s)                 # s dy + y ds = -r_s
    K[isl:, isl:] = np.diag(it.y)
    rhs = -np.concatenate([rd, rp, rl, ru, rs])
    sol = np.linalg.solve(K, rhs)
    np.testing.assert_allclose(d.x, sol[ix:iy], rtol=1e-9, atol=1e-10 * np.abs(sol).max())
    np.testing.assert_allclose(d.y, sol[iy:izl], rtol=1e-9, atol=1e-10 * np.abs(sol).max())
    np.testing.assert_allclose(d.zl, sol[izl:izu], rtol=1e-9, atol=1e-10 * np.abs(sol).max())
    np.testing.assert_allclose(d.zu, sol[izu:isl], rtol=1e-9, atol=1e-10 * np.abs(sol).max())
    np.testing.assert_allclose(d.s, sol[isl:], rtol=1e-9, atol=1e-10 * np.abs(sol).max())


def test_newton_direction_matches_paper_two_sided_system():
    """The paper's own 5x5 system (eq:newton_system, as printed, for l_A <= A x <= u_A with
    residuals r_H = Hx + p - A^T lam_l + A^T lam_u, r_l = A x - s_l - l, r_u = -A x - s_u + u,
    r_c = lam o s - mu) gives the same step as the oracle run on the one-sided stacking
    [A; -A] x <= [u_A; -l_A], with y = (lam_u, lam_l) and s = (s_u, s_l)."""
    rng = np.random.default_rng(7)
    n, mA = 9, 5
    p = _rand_qp(n, mA, 31, cond=1e2)
    A, H, c = p["A"], p["H"], p["c"]
    x = rng.normal(size=n) * 0.3
    lA, uA = A @ x - rng.uniform(0.2, 1, mA), A @ x + rng.uniform(0.2, 1, mA)
    sl, su = rng.uniform(0.1, 2, mA), rng.uniform(0.1, 2, mA)
    ll, lu = rng.uniform(0.1, 2, mA), rng.uniform(0.1, 2, mA)
    mu = 0.05
    # paper form
    rH = H @ x + c - A.T @ ll + A.T @ lu
    rl = A @ x - sl - lA
    ru = -A @ x - su + uA
    rc1, rc2 = ll * sl - mu, lu * su - mu
    N = n + 4 * mA
    K = np.zeros((N, N))
    o = np.cumsum([0, n, mA, mA, mA, mA])
    K[o[0]:o[1], o[0]:o[1]] = H
    K[o[0]:o[1], o[1]:o[2]] = -A.T
    K[o[0]:o[1], o[2]:o[3]] = A.T
    K[o[1]:o[2], o[0]:o[1]] = A
    K[o[1]:o[2], o[3]:o[4]] = -np.eye(mA)
    K[o[2]:o[3], o[0]:o[1]] = -A
    K[o[2]:o[3], o[4]:o[5]] = -np.eye(mA)
    K[o[3]:o[4], o[1]:o[2]] = np.diag(sl)
    K[o[3]:o[4], o[3]:o[4]] = np.diag(ll)
    K[o[4]:o[5], o[2]:o[3]] = np.diag(su)
    K[o[4]:o[5], o[4]:o[5]] = np.diag(lu)
    sol = np.linalg.solve(K, -np.concatenate([rH, rl, ru, rc1, rc2]))
    dx_p, dll, dlu, dsl, dsu = (sol[o[i]:o[i + 1]] for i in range(5))
    # oracle on the one-sided stacking, no variable bounds
    q1 = dict(H=H, c=c, A=np.vstack([A, -A]), b=np.concatenate([uA, -lA]),
              l=np.full(n, -np.inf), u=np.full(n, np.inf))
    it = ipm.Iterate(x, np.concatenate([su, sl]), np.concatenate([lu, ll]), np.zeros(n), np.zeros(n))
    d = ipm.newton_direction(ipm.from_dense(q1), it, mu)
    np.testing.assert_allclose(d.x, dx_p, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(d.y, np.concatenate([dlu, dll]), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(d.s, np.concatenate([dsu, dsl]), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_doubly_augmented_matches_condensed(seed):
    """The paper's doubly augmented form (eq:2x2_augmented) and the condensed form give the
    same (dx, dy)."""
    p = _rand_qp(10, 8, 40 + seed, cond=1e3, free_frac=0.2)
    qp = ipm.from_dense(p)
    it = _interior_point(p, 50 + seed, spread=1.5)
    d = ipm.newton_direction(qp, it, 0.2)
    dx, dy = ipm.doubly_augmented_direction(qp, it, 0.2)
    np.testing.assert_allclose(d.x, dx, rtol=1e-8, atol=1e-10 * np.abs(dx).max())
    np.testing.assert_allclose(d.y, dy, rtol=1e-8, atol=1e-10 * np.abs(dy).max())


# ---------------------------------------------------------------- steps, invariants, identities

def test_step_lengths_reach_boundary():
    """alpha = tau * (largest feasible step): at alpha / tau some component sits on zero and
    none is negative; a step with no blocking component is capped at 1."""
    rng = np.random.default_rng(3)
    n, m = 30, 20
    p = _rand_qp(n, m, 9, free_frac=0.3)
    qp = ipm.from_dense(p)
    it = _interior_point(p, 4)
    d = ipm.Iterate(rng.normal(size=n), rng.normal(size=m) * 3, rng.normal(size=m) * 3,
                    rng.normal(size=n) * 3, rng.normal(size=n) * 3)
    tau = 0.9
    ap, ad = ipm.step_lengths(qp, it, d, tau)
    assert 0 < ap < 1 and 0 < ad < 1
    fl, fu = qp.fl, qp.fu
    xs = it.x + ap / tau * d.x
    prim = np.concatenate([it.s + ap / tau * d.s, (xs - qp.l)[fl], (qp.u - xs)[fu]])
    dual = np.concatenate([it.y + ad / tau * d.y, (it.zl + ad / tau * d.zl)[fl], (it.zu + ad / tau * d.zu)[fu]])
    assert prim.min() > -1e-12 and abs(prim.min()) < 1e-12
    assert dual.min() > -1e-12 and abs(dual.min()) < 1e-12
    up = ipm.Iterate(np.zeros(n), np.abs(d.s), np.abs(d.y), np.abs(d.zl), np.abs(d.zu))
    assert ipm.step_lengths(qp, it, up, tau) == (1.0, 1.0)


def test_iterates_stay_interior_and_gap_identity():
    """Every oracle iterate keeps s, y, t_l, t_u, z_l, z_u > 0 (Section 3.1 line search), and at
    any primal-dual feasible point pobj - dobj = s^T y + t_l^T z_l + t_u^T z_u."""
    p = W.dense_qp(n=80, m=120, seed=5)
    qp = ipm.from_dense(p)
    it, info = ipm.solve(qp, tol=1e-9, record=True)
    assert info.status == "optimal"
    assert min(h["min_pos"] for h in info.history if "min_pos" in h) > 0
    # feasible point: choose x, s, y, z, then define b and c so that r_p = r_d = 0
    rng = np.random.default_rng(1)
    n, m = 15, 9
    q = _rand_qp(n, m, 77, free_frac=0.3)
    x, s, y, zl, zu = W.random_iterate(n, m, q["l"], q["u"], 5)
    q["b"] = q["A"] @ x + s
    q["c"] = -(q["H"] @ x + q["A"].T @ y - zl + zu)
    ops = kkt_check.dense_ops(q)
    val, det = kkt_check.rel_kkt(ops, x, y, zl, zu, detail=True)
    fl, fu = np.isfinite(q["l"]), np.isfinite(q["u"])
    comp = s @ y + np.sum((x - q["l"])[fl] * zl[fl]) + np.sum((q["u"] - x)[fu] * zu[fu])
    assert abs((det["pobj"] - det["dobj"]) - comp) < 1e-10 * (1 + abs(comp))
    assert det["primal"] == 0.0 and det["dual"] < 1e-14


def test_checker_rt_operators_match_dense():
    """The checker's sparse RT operators agree with the dense expansion of the same QP."""
    p = W.rt_qp(n=300, seed=2)
    qp = ipm.from_rt(p)
    ops = kkt_check.rt_ops(p)
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=p["n"]), rng.normal(size=p["m"])
    np.testing.assert_allclose(ops.Hx(x), qp.H @ x, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(ops.Ax(x), qp.A @ x, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(ops.Aty(y), qp.A.T @ y, rtol=1e-12, atol=1e-10)


def test_oracle_solves_small_rt_and_dense():
    """End-to-end oracle runs certify in the independent checker."""
    p = W.rt_qp(n=400, seed=4)
    it, info = ipm.solve(ipm.from_rt(p), tol=1e-9)
    assert info.status == "optimal"
    assert kkt_check.rel_kkt(kkt_check.rt_ops(p), it.x, it.y, it.zl, it.zu) < 1e-8
    p = W.dense_qp(n=100, m=200, seed=8)
    it, info = ipm.solve(ipm.from_dense(p), tol=1e-9)
    assert info.status == "optimal"
    assert kkt_check.rel_kkt(kkt_check.dense_ops(p), it.x, it.y, it.zl, it.zu) < 1e-8


def test_checker_sampled_entries_match_dense():
    """The one-entry-at-a-time operator evaluation used at full size equals the dense
    condensed matrix of the oracle applied to the same vector."""
    p = W.rt_qp(n=250, seed=6)
    qp = ipm.from_rt(p)
    it = ipm.Iterate(*W.random_iterate(p["n"], p["m"], p["l"], p["u"], 3, 1.0))
    res = ipm.residuals(qp, it, 0.1)
    K, _, _, _ = ipm.condensed_system(qp, it, res)
    pv = np.random.default_rng(2).normal(size=p["n"])
    cols = np.array([0, 7, 100, 249])
    q = kkt_check.rt_condensed_entries(p, it.x, it.s, it.y, it.zl, it.zu, pv, cols)
    np.testing.assert_allclose(q, (K @ pv)[cols], rtol=1e-11)
    rd = kkt_check.rt_residual_dual(p, it.x, it.y, it.zl, it.zu)
    np.testing.assert_allclose(rd, res[0], rtol=1e-11, atol=1e-9)


def test_bfgs_compact_form_equals_dense_recursion():
    """The quasi-Newton Hessian of Section 3.3 (eq:bfgs_hessian) in compact form H0 + U W U^T
    against the BFGS recursion carried out on dense matrices; secant condition; definiteness."""
    p = W.bfgs_qp(n=60, k=7, m_ub=5, m_lb=3, density=0.2, seed=9)
    qp = ipm.from_bfgs(p)
    Hd = np.diag(p["h0"])
    for i in range(p["k"]):
        s = p["S"][:, i]
        y = p["lam"] * s
        Hs = Hd @ s
        Hd = Hd - np.outer(Hs, Hs) / (s @ Hs) + np.outer(y, y) / (y @ s)
    np.testing.assert_allclose(qp.H, Hd, rtol=1e-12, atol=1e-12 * np.abs(Hd).max())
    s_last = p["S"][:, -1]
    np.testing.assert_allclose(qp.H @ s_last, p["lam"] * s_last, rtol=1e-10, atol=1e-13)
    assert np.linalg.eigvalsh(qp.H).min() > 0
    # constraints: upper rows G x <= 1.2 G 1, lower rows -G x <= -0.8 G 1; x = 1 strictly feasible
    assert np.all(qp.A @ np.ones(p["n"]) < qp.b)
    assert np.all(qp.b[:5] > 0) and np.all(qp.b[5:] < 0)


def test_bfgs_qp_solution_kkt():
    """Oracle solve of a small quasi-Newton QP satisfies the checker's KKT conditions and the
    optimality of a bounds-only problem with a positive definite H (x >= 0)."""
    p = W.bfgs_qp(n=40, k=4, seed=2)
    qp = ipm.from_bfgs(p)
    it, info = ipm.solve(qp, tol=1e-10)
    assert info.status == "optimal"
    rk = kkt_check.rel_kkt(kkt_check.bfgs_ops(p), it.x, it.y, it.zl, it.zu)
    assert rk <= 1e-9
    g = qp.H @ it.x + qp.c        # x >= 0: g >= 0 where x = 0, g = 0 where x > 0
    act = it.x < 1e-7
    assert np.all(g[act] >= -1e-6) and np.abs(g[~act]).max() <= 1e-6 * (1 + np.abs(qp.c).max())


def test_bfgs_checker_operators_match_dense_form():
    """The checker's matrix-free quasi-Newton operators against the dense H, A of the
    (separately pinned) dense form."""
    p = W.bfgs_qp(n=50, k=5, m_ub=7, m_lb=4, density=0.2, seed=12)
    qp = ipm.from_bfgs(p)
    ops = kkt_check.bfgs_ops(p)
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=p["n"]), rng.normal(size=p["m"])
    np.testing.assert_allclose(ops.Hx(x), qp.H @ x, rtol=1e-12, atol=1e-12 * np.abs(qp.H).max())
    np.testing.assert_allclose(ops.Ax(x), qp.A @ x, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(ops.Aty(y), qp.A.T @ y, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- two-sided rows

def _two_sided_case(n, m, seed, inf_frac=0.25):
    """Random two-sided rows around a feasible point: windows bl < A x_f < bu, with some
    sides (never both of a row) at infinity."""
    p = _rand_qp(n, m, seed, free_frac=0.2)
    rng = np.random.default_rng(500 + seed)
    xf = rng.uniform(-0.4, 0.4, size=n)
    Ax = p["A"] @ xf
    bu = Ax + rng.uniform(0.05, 0.6, size=m)
    bl = Ax - rng.uniform(0.05, 0.6, size=m)
    drop = rng.random(m) < inf_frac
    side = rng.random(m) < 0.5
    bu[drop & side] = np.inf
    bl[drop & ~side] = -np.inf
    p["bl"], p["b"] = bl, bu
    return p


def test_two_sided_single_variable_rows_closed_form():
    """Diagonal H with rows a_k x_{j_k} (distinct j_k, both signs of a_k): every variable's
    window is the intersection of its bounds and its row's [bl/a, bu/a] (flipped for a < 0),
    so x_j = clip(-c_j / h_j, window) and, where the row side is the binding one, the row's
    signed multiplier is -(h_j x_j + c_j) / a_k."""
    rng = np.random.default_rng(77)
    n, m = 30, 20
    h = 10 ** rng.uniform(-1, 1, size=n)
    c = rng.normal(size=n) * 3
    l = np.full(n, -4.0)
    u = np.full(n, 4.0)
    cols = rng.permutation(n)[:m]
    a = rng.uniform(0.5, 2.0, size=m) * np.where(rng.random(m) < 0.5, -1.0, 1.0)
    A = np.zeros((m, n))
    A[np.arange(m), cols] = a
    bl = rng.uniform(-1.5, -0.2, size=m)
    bu = rng.uniform(0.2, 1.5, size=m)
    bl[:3] = -np.inf
    bu[3:6] = np.inf
    lo, hi = l.copy(), u.copy()
    for k, j in enumerate(cols):
        r1, r2 = bl[k] / a[k], bu[k] / a[k]
        rlo, rhi = (r1, r2) if a[k] > 0 else (r2, r1)
        lo[j] = max(lo[j], rlo)
        hi[j] = min(hi[j], rhi)
    x_star = np.clip(-c / h, lo, hi)
    qp, up, lw = ipm.two_sided(np.diag(h), c, A, bl, bu, l, u)
    it, info = ipm.solve(qp, tol=1e-12)
    assert info.status == "optimal"
    np.testing.assert_allclose(it.x, x_star, rtol=1e-8, atol=1e-9)
    y = ipm.row_multipliers(it.y, up, lw, m)
    for k, j in enumerate(cols):
        g = h[j] * x_star[j] + c[j]
        at_row = (x_star[j] == lo[j] and lo[j] > l[j]) or (x_star[j] == hi[j] and hi[j] < u[j])
        want = -g / a[k] if at_row else 0.0
        assert abs(y[k] - want) <= 1e-7 * (1 + abs(want)), (k, y[k], want)
    p = dict(H=np.diag(h), c=c, A=A, b=bu, bl=bl, l=l, u=u)
    assert kkt_check.rel_kkt(kkt_check.dense_ops(p), it.x, y, it.zl, it.zu) < 1e-11


@pytest.mark.parametrize("n,m,seed", [(2, 2, 0), (3, 2, 1), (4, 3, 2), (5, 3, 3), (4, 4, 4)])
def test_two_sided_bruteforce(n, m, seed):
    """Three states per row (inactive, at bu, at bl) and per variable: the oracle on the
    stacked rows [A; -A] reaches the enumerated optimum, its signed row multipliers match the
    enumerated ones, and both points certify in the checker's two-sided mode."""
    p = _two_sided_case(n, m, seed)
    bf = solve_bruteforce_two_sided(p["H"], p["c"], p["A"], p["bl"], p["b"], p["l"], p["u"])
    assert bf is not None
    f, xb, yb, zlb, zub = bf
    qp, up, lw = ipm.two_sided(p["H"], p["c"], p["A"], p["bl"], p["b"], p["l"], p["u"])
    it, info = ipm.solve(qp, tol=1e-12)
    assert info.status == "optimal"
    np.testing.assert_allclose(it.x, xb, atol=1e-8)
    y = ipm.row_multipliers(it.y, up, lw, m)
    np.testing.assert_allclose(y, yb, atol=1e-6 * (1 + np.abs(yb).max()))
    ops = kkt_check.dense_ops(p)
    assert kkt_check.rel_kkt(ops, xb, yb, zlb, zub) < 1e-12
    assert kkt_check.rel_kkt(ops, it.x, y, it.zl, it.zu) < 1e-11


def test_two_sided_stack_matches_paper_newton_system():
    """ipm.two_sided's stack, at the paper's variables of eq:newton_system (stacked as
    y = (lam_u, lam_l), s = (s_u, s_l)), gives the step of the paper's own 5x5 system."""
    rng = np.random.default_rng(8)
    n, mA = 7, 4
    p = _rand_qp(n, mA, 32, cond=1e2)
    A, H, c = p["A"], p["H"], p["c"]
    x = rng.normal(size=n) * 0.3
    lA, uA = A @ x - rng.uniform(0.2, 1, mA), A @ x + rng.uniform(0.2, 1, mA)
    sl, su = rng.uniform(0.1, 2, mA), rng.uniform(0.1, 2, mA)
    ll, lu = rng.uniform(0.1, 2, mA), rng.uniform(0.1, 2, mA)
    mu = 0.03
    N = n + 4 * mA
    K = np.zeros((N, N))
    o = np.cumsum([0, n, mA, mA, mA, mA])
    K[o[0]:o[1], o[0]:o[1]] = H
    K[o[0]:o[1], o[1]:o[2]] = -A.T
    K[o[0]:o[1], o[2]:o[3]] = A.T
    K[o[1]:o[2], o[0]:o[1]] = A
    K[o[1]:o[2], o[3]:o[4]] = -np.eye(mA)
    K[o[2]:o[3], o[0]:o[1]] = -A
    K[o[2]:o[3], o[4]:o[5]] = -np.eye(mA)
    K[o[3]:o[4], o[1]:o[2]] = np.diag(sl)
    K[o[3]:o[4], o[3]:o[4]] = np.diag(ll)
    K[o[4]:o[5], o[2]:o[3]] = np.diag(su)
    K[o[4]:o[5], o[4]:o[5]] = np.diag(lu)
    rhs = np.concatenate([H @ x + c - A.T @ ll + A.T @ lu, A @ x - sl - lA, -A @ x - su + uA,
                          ll * sl - mu, lu * su - mu])
    sol = np.linalg.solve(K, -rhs)
    qp, up, lw = ipm.two_sided(H, c, A, lA, uA, np.full(n, -np.inf), np.full(n, np.inf))
    assert list(up) == list(range(mA)) and list(lw) == list(range(mA))
    it = ipm.Iterate(x, np.concatenate([su, sl]), np.concatenate([lu, ll]), np.zeros(n), np.zeros(n))
    d = ipm.newton_direction(qp, it, mu)
    np.testing.assert_allclose(d.x, sol[o[0]:o[1]], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(d.y, np.concatenate([sol[o[2]:o[3]], sol[o[1]:o[2]]]), rtol=1e-10, atol=1e-12)


def test_checker_two_sided_catches_wrong_sign_and_lower_violation():
    """The checker's two-sided mode: the enumerated KKT point scores ~0, the same point with
    its row multipliers negated fails the dual part, and a point below a finite lower side
    fails the primal part (planted mistakes on the CPU)."""
    p = _two_sided_case(4, 3, 11, inf_frac=0.0)
    f, xb, yb, zlb, zub = solve_bruteforce_two_sided(p["H"], p["c"], p["A"], p["bl"], p["b"], p["l"], p["u"])
    ops = kkt_check.dense_ops(p)
    assert kkt_check.rel_kkt(ops, xb, yb, zlb, zub) < 1e-12
    assert np.abs(yb).max() > 1e-3, "the case needs an active row"
    assert kkt_check.rel_kkt(ops, xb, -yb, zlb, zub) > 1e-4
    k = int(np.argmax(np.abs(p["A"]).sum(axis=1)))
    x_bad = xb - p["A"][k] * ((p["A"][k] @ xb - p["bl"][k]) + 0.5) / (p["A"][k] @ p["A"][k])
    val, parts = kkt_check.rel_kkt(ops, x_bad, yb, zlb, zub, detail=True)
    assert parts["primal"] >= 0.5 / (1 + max(np.abs(p["b"]).max(), np.abs(p["bl"]).max())) - 1e-12


# ---------------------------------------------------------------- readings: invariants

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_start_point_strictly_interior(seed):
    """The start point (a reading: the paper only asks for positive slacks) is strictly
    inside every finite bound, with s, y and the finite-bound z positive and mu0 their mean
    complementarity; z is zero at infinite bounds."""
    p = _rand_qp(12, 7, 300 + seed, free_frac=0.5)
    qp = ipm.from_dense(p)
    it, mu0 = ipm.start_point(qp)
    fl, fu = qp.fl, qp.fu
    assert np.all(it.x[fl] > qp.l[fl]) and np.all(it.x[fu] < qp.u[fu])
    assert np.all(it.s > 0) and np.all(it.y > 0)
    assert np.all(it.zl[fl] > 0) and np.all(it.zu[fu] > 0)
    assert np.all(it.zl[~fl] == 0) and np.all(it.zu[~fu] == 0)
    pairs = np.concatenate([it.s * it.y, (it.x - qp.l)[fl] * it.zl[fl], (qp.u - it.x)[fu] * it.zu[fu]])
    assert mu0 == pytest.approx(pairs.mean(), rel=1e-14)


def test_mu_test_norm_vanishes_only_on_the_central_path():
    """The mu test's ||r|| (a reading: the paper leaves the norm open) is zero at a point
    that is primal and dual feasible with every complementarity product equal to mu, and
    positive as soon as one residual block (r_p, r_d, r_s, r_l, r_u) is planted."""
    n, m, mu = 10, 6, 0.3
    q = _rand_qp(n, m, 55)
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.5, 0.5, size=n)
    s = rng.uniform(0.2, 2.0, size=m)
    y = mu / s
    zl, zu = mu / (x - q["l"]), mu / (q["u"] - x)
    q["b"] = q["A"] @ x + s
    q["c"] = -(q["H"] @ x + q["A"].T @ y - zl + zu)
    qp = ipm.from_dense(q)
    it = ipm.Iterate(x, s, y, zl, zu)
    assert ipm.scaled_residual_norm(qp, it, ipm.residuals(qp, it, mu)) < 1e-13
    for k in range(5):
        res = list(ipm.residuals(qp, it, mu))
        res[k] = res[k].copy()
        res[k][0] += 1e-3
        assert ipm.scaled_residual_norm(qp, it, tuple(res)) > 1e-6, k
