"""GPU parity: every step of the device IPM against the CPU oracle, through the C ABI.

Sizes span several blocks of every kernel and leave ragged tails (n, m not multiples of the
warp or block size).  Floating-point tolerances follow from FP64 arithmetic with a different
summation order: elementwise 1e-10 relative for single products and residuals; PCG
directions within their requested tolerance; end-to-end results at the accuracy bar of
relative KKT <= tol and relative objective difference <= 1e-6 against the oracle.
"""
import numpy as np
import pytest

from oracle import ipm as O
from oracle import kkt_check
from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_03584_gb300 import build
    build.build()
    ipm.load()


def _dense_problem(n, m, seed, free_frac=0.0):
    p = W.dense_qp(n=n, m=m, seed=seed)
    rng = np.random.default_rng(seed + 100)
    if free_frac:
        f = rng.random(n) < free_frac
        p["l"] = np.where(f & (rng.random(n) < 0.5), -np.inf, p["l"])
        p["u"] = np.where(f & (rng.random(n) < 0.5), np.inf, p["u"])
    return p


def _load(p, **opts):
    s = ipm.Solver(**opts)
    if p.get("kind") == "rt":
        s.set_qp_rt(p)
        qp = O.from_rt(p)
    else:
        s.set_qp_dense(p["H"], p["c"], p["A"], p["b"], p["l"], p["u"])
        qp = O.from_dense(p)
    return s, qp


def _iterate(p, qp, seed, spread=1.0):
    x, sl, y, zl, zu = W.random_iterate(qp.n, qp.m, qp.l, qp.u, seed, spread)
    return O.Iterate(x, sl, y, zl, zu)


CASES = [
    ("dense_37x53", lambda: _dense_problem(37, 53, 1, free_frac=0.3)),
    ("dense_300x700", lambda: _dense_problem(300, 700, 2)),
    ("rt_1237", lambda: W.rt_qp(n=1237, seed=3)),
    ("rt_box_only", lambda: dict(W.rt_qp(n=517, seed=4), m=0, a_rows=np.zeros(0, np.int32), b=np.zeros(0))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_residuals_operator_diag(name, make):
    p = make()
    s, qp = _load(p, precond="jacobi")
    it = _iterate(p, qp, 7, spread=1.5)
    mu = 0.37
    s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, mu)
    r = s.residuals()
    rd, rp, rs, rl, ru = O.residuals(qp, it, mu)
    tol = lambda v: 1e-11 * (1 + np.abs(v).max())
    np.testing.assert_allclose(r["rd"], rd, rtol=1e-10, atol=tol(rd))
    np.testing.assert_allclose(r["rp"], rp, rtol=1e-10, atol=tol(rp) if rp.size else 0)
    np.testing.assert_allclose(r["rs"], rs, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["rl"], rl, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["ru"], ru, rtol=1e-12, atol=1e-14)
    ops = kkt_check.rt_ops(p) if p.get("kind") == "rt" else kkt_check.dense_ops(p)
    val, det = kkt_check.rel_kkt(ops, it.x, it.y, it.zl, it.zu, detail=True)
    assert abs(r["dual"] - det["dual"]) <= 1e-10 * (1 + det["dual"])
    assert abs(r["gap"] - det["gap"]) <= 1e-10 * (1 + det["gap"])
    # operator apply q = (H + A^T Theta A + Sigma) p and its Jacobi diagonal
    K, _, _, _ = O.condensed_system(qp, it, (rd, rp, rs, rl, ru))
    rng = np.random.default_rng(5)
    for _ in range(2):
        pv = rng.normal(size=qp.n)
        q = s.apply_kkt(pv)
        ref = K @ pv
        np.testing.assert_allclose(q, ref, rtol=1e-10, atol=1e-12 * np.abs(K).max() * np.abs(pv).max() * qp.n)
    np.testing.assert_allclose(s.precond_diag(), np.diag(K), rtol=1e-11)
    s.close()


@pytest.mark.parametrize("precond", ["jacobi", "jacobi_lr", "dense", "block32"])
@pytest.mark.parametrize("name,make", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_newton_direction_and_steps(name, make, precond):
    p = make()
    s, qp = _load(p, precond=precond, max_cg=20000)
    it = _iterate(p, qp, 11, spread=1.0)
    mu = 0.05
    s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, mu)
    d = s.newton_direction(eta=1e-12)
    ref = O.newton_direction(qp, it, mu)
    rep = d["report"]
    assert rep["converged"] == 1, rep
    if precond == "dense":
        # the factor of the whole condensed matrix (double-float pairs, about 48 bits) leaves
        # PCG a few iterations to 1e-12; more would mean a broken factor or solve
        assert rep["iters"] <= 4, rep
    # dx: PCG stops at ||r|| <= 1e-12 ||rhs||; the error is bounded by cond(K) times that
    K, rhs, _, _ = O.condensed_system(qp, it, O.residuals(qp, it, mu))
    res = np.linalg.norm(K @ d["dx"] - rhs) / np.linalg.norm(rhs)
    assert res <= 1e-10, res
    scale = lambda v: np.abs(v).max() + 1e-300
    err = lambda a, b: np.abs(a - b).max() / scale(b)
    assert err(d["dx"], ref.x) <= 1e-7
    if qp.m:
        assert err(d["ds"], ref.s) <= 1e-7 and err(d["dy"], ref.y) <= 1e-7
    assert err(d["dzl"], ref.zl) <= 1e-7 and err(d["dzu"], ref.zu) <= 1e-7
    # ratio test on the oracle's direction: same candidates, same minimum
    for tau in (0.995, 0.5):
        ap, ad = s.step_lengths(ref.x, ref.s, ref.y, ref.zl, ref.zu, tau)
        ap0, ad0 = O.step_lengths(qp, it, ref, tau)
        assert ap == pytest.approx(ap0, rel=1e-13) and ad == pytest.approx(ad0, rel=1e-13)
    s.close()


def test_dense_preconditioner_from_csr_rows():
    """R too large to keep densely (nR n above 2^25 entries): the dense preconditioner forms
    K from R's CSR rows (one pass over the rows per tile) instead of the dense copy; the
    Newton direction and its PCG iteration count as with the dense copy."""
    p = W.rt_qp(n=300, V=120_000, density=0.02, seed=8)
    assert p["V"] * p["n"] > (32 << 20)
    s, qp = _load(p, precond="dense", max_cg=20000)
    it = _iterate(p, qp, 12, spread=1.0)
    mu = 0.05
    s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, mu)
    d = s.newton_direction(eta=1e-12)
    rep = d["report"]
    assert rep["converged"] == 1 and rep["iters"] <= 4, rep
    ref = O.newton_direction(qp, it, mu)
    err = lambda a, b: np.abs(a - b).max() / (np.abs(b).max() + 1e-300)
    assert err(d["dx"], ref.x) <= 1e-7 and err(d["dy"], ref.y) <= 1e-7
    s.close()


def _solve_both(p, tol, **opts):
    s, qp = _load(p, tol_kkt=tol, **opts)
    st = s.solve()
    out = s.get()
    s.close()
    ref, info = O.solve(qp, tol=tol)
    assert info.status == "optimal"
    return st, out, ref, qp


def _check_solution(p, qp, st, out, ref, tol):
    assert st == ipm.IPM_OK, out["info"]
    ops = kkt_check.rt_ops(p) if p.get("kind") == "rt" else kkt_check.dense_ops(p)
    rk = kkt_check.rel_kkt(ops, out["x"], out["y"], out["zl"], out["zu"])
    assert rk <= tol * 1.0001, rk
    f = O.objective(qp, out["x"])
    f_ref = O.objective(qp, ref.x)
    assert abs(f - f_ref) / (1 + abs(f_ref)) <= 1e-6
    # x* is unique (H positive definite); its accuracy follows the KKT tolerance
    assert np.abs(out["x"] - ref.x).max() / (1 + np.abs(ref.x).max()) <= 1e-3


@pytest.mark.parametrize("precond", ["dense", "jacobi_lr"])
def test_solve_dense_c0_shape(precond):
    """The dense workload at full size (n = 500, m = 1000, seed 0), tolerance 1e-8."""
    p = W.dense_qp()
    st, out, ref, qp = _solve_both(p, 1e-8, precond=precond, max_cg=20000)
    _check_solution(p, qp, st, out, ref, 1e-8)


@pytest.mark.parametrize("precond", ["jacobi_lr", "dense", "jacobi", "block32"])
def test_solve_rt_small(precond):
    p = W.rt_qp(n=1500, seed=9)
    st, out, ref, qp = _solve_both(p, 1e-7, precond=precond, max_cg=20000)
    _check_solution(p, qp, st, out, ref, 1e-7)


def test_solve_edge_cases():
    # one variable, box only
    p = dict(H=np.array([[2.0]]), c=np.array([3.0]), A=np.zeros((0, 1)), b=np.zeros(0), l=np.array([-1.0]), u=np.array([1.0]))
    st, out, ref, qp = _solve_both(p, 1e-9, precond="jacobi")
    _check_solution(p, qp, st, out, ref, 1e-9)
    assert out["x"][0] == pytest.approx(-1.0, abs=1e-8)
    # free variables and rows only (no bounds anywhere)
    q = _dense_problem(45, 20, 3)
    q["l"] = np.full(45, -np.inf)
    q["u"] = np.full(45, np.inf)
    st, out, ref, qp = _solve_both(q, 1e-8, precond="jacobi_lr", max_cg=20000)
    _check_solution(q, qp, st, out, ref, 1e-8)
    # RT with an empty voxel row and an empty constraint row (a_rows pointing at it)
    r = W.rt_qp(n=300, seed=12)
    ip, ix, dv = r["D_indptr"].copy(), r["D_indices"], r["D_data"]
    k0 = int(r["a_rows"][0])
    cut = slice(ip[k0], ip[k0 + 1])
    ix = np.delete(ix, cut)
    dv = np.delete(dv, cut)
    ip[k0 + 1:] -= (ip[k0 + 1] - ip[k0])
    r.update(D_indptr=ip, D_indices=ix, D_data=dv)
    st, out, ref, qp = _solve_both(r, 1e-8, precond="jacobi_lr", max_cg=20000)
    _check_solution(r, qp, st, out, ref, 1e-8)


def test_a_rows_equals_csr_rows():
    """The same constraints given as rows of F or as an explicit CSR matrix give the same x."""
    p = W.rt_qp(n=700, seed=13)
    s1 = ipm.Solver(tol_kkt=1e-9, precond="jacobi_lr")
    s1.set_qp_rt(p)
    assert s1.solve() == ipm.IPM_OK
    x1 = s1.get()["x"]
    ip, ix, dv = p["D_indptr"], p["D_indices"], p["D_data"]
    rows = p["a_rows"].astype(np.int64)
    lens = ip[rows + 1] - ip[rows]
    Aip = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    sel = np.concatenate([np.arange(ip[r], ip[r + 1]) for r in rows])
    s2 = ipm.Solver(tol_kkt=1e-9, precond="jacobi_lr")
    s2.set_qp(p["n"], p["m"], p["c"], p["b"], p["l"], p["u"], h0=p["h0"], F=(ip, ix, dv), f_w=p["w"],
              A=(Aip, ix[sel], dv[sel]))
    assert s2.solve() == ipm.IPM_OK
    x2 = s2.get()["x"]
    assert np.abs(x1 - x2).max() <= 1e-6 * (1 + np.abs(x1).max())
    s1.close()
    s2.close()


def test_bitwise_deterministic():
    p = W.rt_qp(n=900, seed=14)
    xs = []
    for _ in range(2):
        with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr") as s:
            s.set_qp_rt(p)
            assert s.solve() == ipm.IPM_OK
            xs.append(s.get()["x"])
    assert np.array_equal(xs[0], xs[1])


def test_autotuned_schedule_solves():
    p = W.rt_qp(n=1100, seed=16)
    with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr", autotune=1) as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK
        out = s.get()
        assert out["info"]["lanes_rows"] in (4, 8, 16, 32) and out["info"]["lanes_cols"] in (4, 8, 16, 32)
        assert kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-8


def test_direct_launch_mode_matches_graphs():
    """use_graphs = 0 runs the same kernels one by one: the same bits as the graph path."""
    p = W.rt_qp(n=600, seed=17)
    xs = []
    for ug in (1, 0):
        with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr", use_graphs=ug) as s:
            s.set_qp_rt(p)
            assert s.solve() == ipm.IPM_OK
            xs.append(s.get()["x"])
    assert np.array_equal(xs[0], xs[1])


def test_warm_start_from_solution():
    p = W.rt_qp(n=800, seed=15)
    with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr") as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK
        it_cold = s.get()["info"]["ipm_iters"]
        assert s.solve(warm=True) == ipm.IPM_OK
        out = s.get()
        assert out["info"]["ipm_iters"] <= it_cold
        rk = kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"])
        assert rk <= 1e-8


def test_bad_inputs_rejected():
    s = ipm.Solver()
    with pytest.raises(ipm.IpmError) as e:
        s.set_qp(3, 0, np.array([1.0, np.nan, 0.0]))
    assert e.value.status == ipm.IPM_ERR_ARG
    with pytest.raises(ipm.IpmError):
        s.set_qp(2, 0, np.zeros(2), l=np.array([1.0, 0.0]), u=np.array([0.0, 1.0]))
    with pytest.raises(ipm.IpmError) as e:
        s.solve()
    assert e.value.status == ipm.IPM_ERR_STATE
    p = W.rt_qp(n=100, seed=1)
    bad = dict(p)
    bad["a_rows"] = p["a_rows"].copy()
    bad["a_rows"][0] = p["V"] + 5
    with pytest.raises(ipm.IpmError):
        s.set_qp_rt(bad)
    s.close()


@pytest.mark.parametrize("refine_mode", [0, 1])
@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_reduced_precision_operator_refined_to_fp64(storage, refine_mode):
    """D and A stored in FP32 / BF16 / FP8-E4M3 with per-row scales, FP32-accumulating PCG,
    FP64 accuracy of each Newton step by refinement passes (refine_mode 0) or by one PCG
    whose residual is replaced by the FP64 one (1): the solve must still match the FP64
    oracle at the accuracy bar (rel KKT <= tol, rel objective difference <= 1e-6)."""
    p = W.rt_qp(n=1400, seed=19)
    st, out, ref, qp = _solve_both(p, 1e-7, precond="jacobi_lr", storage=storage, max_cg=5000,
                                   refine_mode=refine_mode)
    _check_solution(p, qp, st, out, ref, 1e-7)
    assert out["info"]["refine_passes"] >= out["info"]["ipm_iters"]


@pytest.mark.parametrize("refine_mode", [0, 1])
@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_reduced_precision_direction(storage, refine_mode):
    """One refined Newton direction at a random iterate against the oracle's exact one."""
    p = W.rt_qp(n=900, seed=21)
    s, qp = _load(p, precond="jacobi_lr", storage=storage, max_cg=5000, refine_max=30, refine_mode=refine_mode)
    it = _iterate(p, qp, 13, spread=1.0)
    s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, 0.05)
    d = s.newton_direction(eta=1e-10)
    ref = O.newton_direction(qp, it, 0.05)
    assert d["report"]["converged"] == 1, d["report"]
    err = np.abs(d["dx"] - ref.x).max() / np.abs(ref.x).max()
    assert err <= 1e-6, err
    s.close()


def test_async_and_batch_match_sync():
    """ipm_solve_async / ipm_solve_wait and one batched graph launch over several uneven QPs give
    the same bits as solving each QP on its own."""
    probs = [W.rt_qp(n=n, seed=40 + i, density=d, n_organ=n // 2) for i, (n, d) in
             enumerate([(300, 0.01), (777, 0.004), (1200, 0.006), (450, 0.008)])]
    ref = []
    for p in probs:
        with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr") as s:
            s.set_qp_rt(p)
            assert s.solve() == ipm.IPM_OK
            ref.append(s.get()["x"])
    with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr") as s:
        s.set_qp_rt(probs[1])
        s.solve_async()
        assert s.wait() == ipm.IPM_OK
        assert np.array_equal(s.get()["x"], ref[1])
    solvers = []
    for p in probs:
        s = ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr")
        s.set_qp_rt(p)
        solvers.append(s)
    b = ipm.Batch(solvers)
    for rep in range(2):
        assert b.solve() == [ipm.IPM_OK] * len(probs)
        for s, x in zip(solvers, ref):
            assert np.array_equal(s.get()["x"], x)
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("name,make", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_augmented_system_direction(name, make):
    """PCG on the paper's doubly augmented system (Section 4, eq:2x2_augmented) gives the
    oracle's direction of that system, which equals the condensed one."""
    p = make()
    s, qp = _load(p, system="augmented", max_cg=50000)
    it = _iterate(p, qp, 13, spread=1.0)
    mu = 0.05
    s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, mu)
    d = s.newton_direction(eta=1e-12)
    assert d["report"]["converged"] == 1, d["report"]
    dx_ref, dy_ref = O.doubly_augmented_direction(qp, it, mu)
    err = lambda a, b: np.abs(a - b).max() / (np.abs(b).max() + 1e-300)
    assert err(d["dx"], dx_ref) <= 1e-6
    if qp.m:
        assert err(d["dy"], dy_ref) <= 1e-6
    ref = O.newton_direction(qp, it, mu)
    assert err(d["dx"], ref.x) <= 1e-6
    s.close()


@pytest.mark.parametrize("name,make", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_augmented_system_solves(name, make):
    p = make()
    tol = 1e-8
    s, qp = _load(p, system="augmented", tol_kkt=tol, max_cg=50000)
    st = s.solve()
    out = s.get()
    s.close()
    ref, info = O.solve(qp, tol=tol)
    _check_solution(p, qp, st, out, ref, tol)
    f, f0 = O.objective(qp, out["x"]), O.objective(qp, ref.x)
    assert abs(f - f0) <= 1e-6 * (1 + abs(f0))


def test_dense_preconditioner_needs_f64_storage():
    """DENSE is an FP64 factor for the FP64 operator: refused with a reduced-precision
    operator; AUTO then picks JACOBI_LR even for small n."""
    for storage in ("f32", "bf16", "fp8"):
        with pytest.raises(ipm.IpmError):
            ipm.Solver(precond="dense", storage=storage)
    p = W.rt_qp(n=300, seed=2)
    with ipm.Solver(tol_kkt=1e-7, storage="bf16") as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK
        assert s.get()["info"]["precond"] == ipm.PRECOND["jacobi_lr"]


def test_augmented_system_option_checks():
    with pytest.raises(ipm.IpmError):
        ipm.Solver(system="augmented", storage="bf16")
    with pytest.raises(ipm.IpmError):
        ipm.Solver(system="augmented", precond="jacobi_lr")


def _farkas_ok(A, b, l, u, y, zl, zu):
    """y, z >= 0 with A^T y - z_l + z_u = 0 and b^T y - l^T z_l + u^T z_u < 0 (after scaling)."""
    fl, fu = np.isfinite(l), np.isfinite(u)
    zl = np.where(fl, zl, 0.0)
    zu = np.where(fu, zu, 0.0)
    sc = max(np.abs(y).max(initial=0.0), np.abs(zl).max(), np.abs(zu).max())
    y, zl, zu = y / sc, zl / sc, zu / sc
    res = np.abs(A.T @ y - zl + zu).max()
    gap = b @ y - np.where(fl, l, 0.0) @ zl + np.where(fu, u, 0.0) @ zu
    return y.min(initial=0.0) >= -1e-12 and res <= 1e-6 and gap < -1e-6


@pytest.mark.parametrize("case", ["dense_box", "rt_negative_limit"])
def test_primal_infeasibility_detected(case):
    if case == "dense_box":
        n = 7
        A = np.ones((2, n))
        A[1, :3] = 2.0
        b = np.array([-1.0, 5.0])                 # sum(x) <= -1 with 0 <= x <= 1
        l, u = np.zeros(n), np.ones(n)
        s = ipm.Solver(tol_kkt=1e-8)
        s.set_qp_dense(np.eye(n), np.ones(n), A, b, l, u)
    else:
        p = W.rt_qp(n=700, seed=71, b_organ=-0.5)  # dose <= -0.5 with D >= 0, x >= 0
        qp = O.from_rt(p)
        A, b, l, u = qp.A, qp.b, qp.l, qp.u
        s = ipm.Solver(tol_kkt=1e-8)
        s.set_qp_rt(p)
    st = s.solve()
    out = s.get()
    s.close()
    assert st == ipm.IPM_INFEASIBLE_SUSPECTED, out["info"]
    assert out["info"]["ipm_iters"] < 200
    assert _farkas_ok(A, b, l, u, out["y"], out["zl"], out["zu"])
