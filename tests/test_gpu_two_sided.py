"""GPU parity for two-sided rows bl <= A x <= b (the paper's l_A <= A x <= u_A, Section 4
before eq:2x2_reduced), through the C ABI, against the oracle's own stack [A; -A].

Cases: a dense QP with CSR rows (upper-only, lower-only and free rows among the two-sided
ones) and an RT-shaped QP whose window rows are rows of D (a_rows), so that the library
keeps the fused form for upper sides and stores negated copies for lower sides.  Results are
compared as in the one-sided parity tests: x* is unique (H positive definite), the objective
to 1e-6, the certificate checker (two-sided mode, signed multipliers) at the solve tolerance.
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


def _dense_two_sided(n, m, seed):
    """dense_qp (x = 1 strictly feasible) with lower sides bl = A 1 - U(0.1, 1); about 15%
    of the rows lose the upper side, 15% the lower side, and row 0 both."""
    p = W.dense_qp(n=n, m=m, seed=seed)
    rng = np.random.default_rng(seed + 7)
    bl = p["A"] @ np.ones(n) - rng.uniform(0.1, 1.0, size=m)
    k = rng.random(m)
    b = np.where(k < 0.15, np.inf, p["b"])
    bl = np.where((k >= 0.15) & (k < 0.3), -np.inf, bl)
    b[0], bl[0] = np.inf, -np.inf
    p["b"], p["bl"] = b, bl
    return p


def _csr(A):
    rows, cols = np.nonzero(A)
    indptr = np.zeros(A.shape[0] + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=A.shape[0]), out=indptr[1:])
    return indptr, cols.astype(np.int32), A[rows, cols]


def _args(p):
    if p.get("kind") == "rt":
        return dict(n=p["n"], m=p["m"], c=p["c"], b=p["b"], l=p["l"], u=p["u"], h0=p["h0"],
                    F=(p["D_indptr"], p["D_indices"], p["D_data"]), f_w=p["w"], a_rows=p["a_rows"], bl=p["bl"])
    return dict(n=len(p["c"]), m=len(p["b"]), c=p["c"], b=p["b"], l=p["l"], u=p["u"], H_dense=p["H"],
                A=_csr(p["A"]), bl=p["bl"])


def _load(p, **opts):
    s = ipm.Solver(**opts)
    s.set_qp(**_args(p))
    dq = O.from_rt(p) if p.get("kind") == "rt" else O.from_dense(p)
    qp, up, lo = O.two_sided(dq.H, dq.c, dq.A, p["bl"], p["b"], dq.l, dq.u)
    return s, dq, qp, up, lo


def _ops(p):
    return kkt_check.rt_ops(p) if p.get("kind") == "rt" else kkt_check.dense_ops(p)


CASES = [
    ("dense_150x120", lambda: _dense_two_sided(150, 120, 3)),
    ("rt_900", lambda: W.rt_two_sided(W.rt_qp(n=900, seed=21))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_stored_rows_count(name, make):
    p = make()
    s, dq, qp, up, lo = _load(p)
    sz = s.sizes()
    assert sz == dict(n=dq.n, m=p["m"], m_rows=up.size + lo.size)
    s.close()


@pytest.mark.parametrize("system", ["condensed", "augmented"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_solve_matches_oracle(name, make, system):
    p = make()
    tol = 1e-8
    s, dq, qp, up, lo = _load(p, tol_kkt=tol, system=system, max_cg=50000)
    st = s.solve()
    out = s.get()
    s.close()
    assert st == ipm.IPM_OK, out["info"]
    ref, info = O.solve(qp, tol=tol)
    assert info.status == "optimal"
    x = out["x"]
    assert np.abs(x - ref.x).max() / (1 + np.abs(ref.x).max()) <= 1e-4
    f, f0 = O.objective(qp, x), O.objective(qp, ref.x)
    assert abs(f - f0) <= 1e-6 * (1 + abs(f0))
    # signed row multipliers: the checker's two-sided mode, and the binding sides agree
    rk = kkt_check.rel_kkt(_ops(p), x, out["y"], out["zl"], out["zu"])
    assert rk <= tol * 1.0001, rk
    y0 = O.row_multipliers(ref.y, up, lo, p["m"])
    big = np.abs(y0) > 1e-3 * np.abs(y0).max()
    assert big.sum() > 0 and np.all(np.sign(out["y"][big]) == np.sign(y0[big]))
    assert (y0 < 0).any() and (y0 > 0).any(), "the case must bind both sides"
    # slack per caller row: to the upper side, else to the lower side, +inf for a free row
    Ax = dq.A @ x
    fb, fbl = np.isfinite(p["b"]), np.isfinite(p["bl"])
    want = np.where(fb, np.where(fb, p["b"], 0) - Ax, np.where(fbl, Ax - np.where(fbl, p["bl"], 0), np.inf))
    fin = np.isfinite(want)
    assert np.all(np.isinf(out["s"][~fin]))
    np.testing.assert_allclose(out["s"][fin], want[fin], atol=1e-6 * (1 + np.abs(want[fin]).max()))


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_direction_on_stored_rows(name, make):
    """The step-level calls work on the stored rows: at an iterate given in the stacked
    order (upper sides, then lower sides) the PCG direction is the oracle's Newton step."""
    p = make()
    s, dq, qp, up, lo = _load(p, max_cg=50000)
    x, sl, y, zl, zu = W.random_iterate(qp.n, qp.m, qp.l, qp.u, 17, 1.0)
    it = O.Iterate(x, sl, y, zl, zu)
    mu = 0.05
    s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, mu)
    d = s.newton_direction(eta=1e-12)
    assert d["report"]["converged"] == 1, d["report"]
    ref = O.newton_direction(qp, it, mu)
    err = lambda a, b: np.abs(a - b).max() / (np.abs(b).max() + 1e-300)
    assert err(d["dx"], ref.x) <= 1e-7
    assert err(d["dy"], ref.y) <= 1e-7 and err(d["ds"], ref.s) <= 1e-7
    r = s.residuals()
    r0 = O.residuals(qp, it, mu)
    np.testing.assert_allclose(r["rp"], r0[1], rtol=1e-10, atol=1e-10 * (1 + np.abs(r0[1]).max()))
    s.close()


def test_device_inputs_give_identical_result():
    """The same QP from device arrays (the stack is built from copies fetched to the host)
    gives bit-identical results to host arrays."""
    torch = pytest.importorskip("torch")
    p = W.rt_two_sided(W.rt_qp(n=700, seed=23))
    a = _args(p)
    s1 = ipm.Solver(tol_kkt=1e-8)
    s1.set_qp(**a)
    s1.solve()
    o1 = s1.get()
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    ad = {k: (tuple(dev(t) for t in v) if isinstance(v, tuple) else dev(v) if isinstance(v, np.ndarray) else v)
          for k, v in a.items()}
    s2 = ipm.Solver(tol_kkt=1e-8)
    s2.set_qp(**ad)
    s2.solve()
    o2 = s2.get()
    assert np.array_equal(o1["x"], o2["x"]) and np.array_equal(o1["y"], o2["y"])
    assert o1["info"]["ipm_iters"] == o2["info"]["ipm_iters"]
    s1.close()
    s2.close()


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_reduced_precision_two_sided(storage):
    """Reduced-precision operator with FP64 refinement on the stacked rows (the negated
    copies are quantised like every other row): FP64 accuracy at the checker.  The default
    preconditioner is JACOBI_LR here (AUTO keeps the dense factor for FP64 storage)."""
    p = W.rt_two_sided(W.rt_qp(n=900, seed=21))
    tol = 1e-7
    s, dq, qp, up, lo = _load(p, tol_kkt=tol, storage=storage, max_cg=50000)
    st = s.solve()
    out = s.get()
    s.close()
    assert st == ipm.IPM_OK, out["info"]
    assert out["info"]["precond"] == ipm.PRECOND["jacobi_lr"]
    assert kkt_check.rel_kkt(_ops(p), out["x"], out["y"], out["zl"], out["zu"]) <= tol * 1.0001


def test_shared_plan_keeps_row_map():
    """ipm_share_qp of a two-sided plan: the second handle reports the caller's rows too."""
    p = _dense_two_sided(90, 70, 5)
    s1 = ipm.Solver(tol_kkt=1e-8)
    s1.set_qp(**_args(p))
    s2 = ipm.Solver(tol_kkt=1e-8).share_qp(s1)
    assert s2.sizes() == s1.sizes()
    s1.solve()
    s2.solve()
    o1, o2 = s1.get(), s2.get()
    assert np.array_equal(o1["x"], o2["x"]) and np.array_equal(o1["y"], o2["y"])
    assert np.array_equal(o1["s"], o2["s"])
    s2.close()
    s1.close()


def test_bad_row_bounds_rejected():
    p = _dense_two_sided(20, 10, 6)
    for bad in ("cross", "equal", "nan", "neg_inf_upper", "pos_inf_lower"):
        q = dict(p)
        b, bl = p["b"].copy(), p["bl"].copy()
        if bad == "cross":
            b[3], bl[3] = 0.0, 1.0
        elif bad == "equal":
            b[3], bl[3] = 0.5, 0.5
        elif bad == "nan":
            bl[4] = np.nan
        elif bad == "neg_inf_upper":
            b[5] = -np.inf
        else:
            bl[6] = np.inf
        q["b"], q["bl"] = b, bl
        s = ipm.Solver()
        with pytest.raises(ipm.IpmError):
            s.set_qp(**_args(q))
        s.close()
    # one-sided rows still need finite b
    q = dict(p)
    q["b"], q["bl"] = p["b"].copy(), None
    q["b"][2] = np.inf
    s = ipm.Solver()
    with pytest.raises(ipm.IpmError):
        s.set_qp(**_args(q))
    s.close()


def test_all_rows_free():
    """Rows with neither side finite drop out: the QP is the bounds-only one (bit-identical
    solution), y = 0 and s = +inf for every caller row."""
    p = _dense_two_sided(40, 12, 9)
    p["b"], p["bl"] = np.full(12, np.inf), np.full(12, -np.inf)
    with ipm.Solver(tol_kkt=1e-8) as s1:
        s1.set_qp(**_args(p))
        assert s1.sizes()["m_rows"] == 0
        assert s1.solve() == ipm.IPM_OK
        o1 = s1.get()
    with ipm.Solver(tol_kkt=1e-8) as s2:
        s2.set_qp(n=40, m=0, c=p["c"], l=p["l"], u=p["u"], H_dense=p["H"])
        assert s2.solve() == ipm.IPM_OK
        o2 = s2.get()
    assert np.array_equal(o1["x"], o2["x"])
    assert np.all(o1["y"] == 0) and np.all(np.isinf(o1["s"]))


def test_duplicate_a_rows_rejected():
    """As for one-sided rows, a row of F may be named once (its two sides are bl and b)."""
    p = W.rt_two_sided(W.rt_qp(n=300, seed=4))
    q = dict(p)
    q["a_rows"] = p["a_rows"].copy()
    q["a_rows"][-1] = q["a_rows"][-2]
    s = ipm.Solver()
    with pytest.raises(ipm.IpmError) as e:
        s.set_qp(**_args(q))
    assert e.value.status == ipm.IPM_ERR_ARG
    s.close()
