"""The PCG operator's arithmetic (float64 or double-float) and the format of its rows pass
(CSR or runs) on every problem family, against the CPU oracle: whole solves at the accuracy
bar (checker rel. KKT <= tol, relative objective difference <= 1e-6 against the oracle's),
bitwise reproducibility, the graph and direct-launch paths, and the fallbacks (double-float
refused for values outside the float32 pair's range; runs not taken by AUTO when rows are
scattered)."""
import numpy as np
import pytest

from oracle import ipm as O
from oracle import kkt_check
from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu

VARIANTS = [("f64", "runs"), ("df32", "csr"), ("df32", "runs"), ("df32", "runs-staged"), ("mixed", "csr")]


def _fmt(fmt):
    """rows_format and rows_stage options of a variant name ("runs-staged": the
    pieces streamed through the shared-memory copy pipeline instead of read from global memory)."""
    return dict(rows_format=fmt.split("-")[0], rows_stage=1 if fmt.endswith("-staged") else 0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_03584_gb300 import build
    build.build()
    ipm.load()


def _check(p, qp, st, out, tol, ops):
    assert st == ipm.IPM_OK, out["info"]
    rk = kkt_check.rel_kkt(ops, out["x"], out["y"], out["zl"], out["zu"])
    assert rk <= tol * 1.0001, rk
    ref, info = O.solve(qp, tol=min(tol, 1e-9))
    assert info.status == "optimal"
    f, f0 = O.objective(qp, out["x"]), O.objective(qp, ref.x)
    assert abs(f - f0) / (1 + abs(f0)) <= 1e-6


@pytest.mark.parametrize("arith,fmt", VARIANTS, ids=["%s-%s" % v for v in VARIANTS])
@pytest.mark.parametrize("precond", ["jacobi_lr", "jacobi"])
def test_rt_solves(arith, fmt, precond):
    p = W.rt_qp(n=1500, seed=9)
    with ipm.Solver(tol_kkt=1e-7, precond=precond, op_arith=arith, **_fmt(fmt), max_cg=20000) as s:
        s.set_qp_rt(p)
        st = s.solve()
        out = s.get()
    assert out["info"]["op_arith"] == ipm.ARITH[arith] and out["info"]["rows_runs"] == fmt.startswith("runs")
    _check(p, O.from_rt(p), st, out, 1e-7, kkt_check.rt_ops(p))


@pytest.mark.parametrize("arith,fmt", VARIANTS, ids=["%s-%s" % v for v in VARIANTS])
def test_dense_h_block_solves(arith, fmt):
    """A dense H block (its FP64 part of the column pass) and dense rows of A (one run each)."""
    p = W.dense_qp(n=300, m=700, seed=2)
    with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr", op_arith=arith, **_fmt(fmt), max_cg=20000) as s:
        s.set_qp_dense(p["H"], p["c"], p["A"], p["b"], p["l"], p["u"])
        st = s.solve()
        out = s.get()
    _check(p, O.from_dense(p), st, out, 1e-8, kkt_check.dense_ops(p))


@pytest.mark.parametrize("arith,fmt", VARIANTS, ids=["%s-%s" % v for v in VARIANTS])
def test_lowrank_hessian_solves(arith, fmt):
    """The quasi-Newton term U W U^T (FP64 inside the double-float column pass) with CSR rows."""
    q = W.bfgs_qp(n=3000, k=20, m_ub=900, m_lb=300, density=0.01, seed=6, c_mode="target", ub_fac=1.1, lb_fac=0.9)
    with ipm.Solver(tol_kkt=1e-7, precond="jacobi_lr", op_arith=arith, **_fmt(fmt), stiff_max=1024) as s:
        s.set_qp_bfgs(q)
        st = s.solve()
        out = s.get()
    qp = O.from_bfgs(q)
    _check(q, qp, st, out, 1e-7, kkt_check.bfgs_ops(q))


@pytest.mark.parametrize("arith,fmt", VARIANTS, ids=["%s-%s" % v for v in VARIANTS])
def test_augmented_and_two_sided_solves(arith, fmt):
    """The paper's doubly augmented system (the rows pass also forms its bottom block) and
    two-sided rows (negated copies of rows appended to R)."""
    p = W.rt_qp(n=900, seed=13)
    with ipm.Solver(tol_kkt=1e-8, system="augmented", op_arith=arith, **_fmt(fmt), max_cg=50000) as s:
        s.set_qp_rt(p)
        st = s.solve()
        out = s.get()
    _check(p, O.from_rt(p), st, out, 1e-8, kkt_check.rt_ops(p))
    t = W.rt_two_sided(W.rt_qp(n=1100, seed=5), n_window=40)
    with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr", op_arith=arith, **_fmt(fmt), stiff_max=1024) as s:
        s.set_qp_rt(t)
        st = s.solve()
        out = s.get()
    assert st == ipm.IPM_OK, out["info"]
    dq = O.from_rt(t)
    qp, _, _ = O.two_sided(dq.H, dq.c, dq.A, t["bl"], t["b"], dq.l, dq.u)
    ref, info = O.solve(qp, tol=1e-9)
    f, f0 = O.objective(qp, out["x"]), O.objective(qp, ref.x)
    assert abs(f - f0) / (1 + abs(f0)) <= 1e-6


@pytest.mark.parametrize("arith,fmt", VARIANTS, ids=["%s-%s" % v for v in VARIANTS])
def test_bitwise_reproducible_and_direct_launches(arith, fmt):
    p = W.rt_qp(n=900, seed=14)
    xs = []
    for ug in (1, 1, 0):
        with ipm.Solver(tol_kkt=1e-8, precond="jacobi_lr", op_arith=arith, **_fmt(fmt), use_graphs=ug) as s:
            s.set_qp_rt(p)
            assert s.solve() == ipm.IPM_OK
            xs.append(s.get()["x"])
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[0], xs[2])


@pytest.mark.parametrize("arith,storage", [("df32", "f64"), ("f64", "bf16"), ("f64", "fp8")])
def test_rows_longer_than_a_stage(arith, storage):
    """Rows whose values do not fit one shared-memory stage of the staged rows pass (64 KB:
    more than 8190 double-float or 32760 BF16 entries) are tiles of their own, read from
    global memory, between ordinary staged tiles.  Against the definition: sampled entries of
    one operator apply (double-float) and a solve certified by the checker (every storage)."""
    p = W.rt_qp(n=40000, V=3000, seed=17, n_organ=300)
    ip, ix, dv = p["D_indptr"], p["D_indices"], p["D_data"]
    rng = np.random.default_rng(2)
    long_rows = {5: (100, 36000), 1700: (2000, 35000), 2999: (0, 40000)}   # row: (first column, length)
    rows_i, rows_d = [], []
    for r in range(p["V"]):
        if r in long_rows:
            c0, ln = long_rows[r]
            rows_i.append(np.arange(c0, c0 + ln, dtype=np.int32))
            rows_d.append(rng.lognormal(0.0, 1.0, ln) * 0.01)
        else:
            rows_i.append(ix[ip[r]:ip[r + 1]])
            rows_d.append(dv[ip[r]:ip[r + 1]])
    q = dict(p)
    q["D_indptr"] = np.concatenate([[0], np.cumsum([len(a) for a in rows_i])]).astype(np.int64)
    q["D_indices"] = np.concatenate(rows_i).astype(np.int32)
    q["D_data"] = np.concatenate(rows_d)
    # the cost keeps its definition c = -D^T W d with the new rows
    rowid = np.repeat(np.arange(q["V"]), np.diff(q["D_indptr"]))
    q["c"] = -np.bincount(q["D_indices"], weights=q["D_data"] * (q["w"] * q["d"])[rowid], minlength=q["n"])
    with ipm.Solver(tol_kkt=1e-6, op_arith=arith, storage=storage, rows_format="runs", rows_stage=1,
                    max_cg=5000) as s:
        s.set_qp_rt(q)
        if storage == "f64":
            x, sl, y, zl, zu = W.random_iterate(q["n"], q["m"], q["l"], q["u"], 3, 1.0)
            s.set_iterate(x, sl, y, zl, zu, 0.1)
            pv = rng.normal(size=q["n"])
            qv = s.apply_kkt(pv)
            cols = np.concatenate([[0, 100, 2000, 39999], rng.choice(q["n"], 60, replace=False)])
            ref = kkt_check.rt_condensed_entries(q, x, sl, y, zl, zu, pv, cols)
            np.testing.assert_allclose(qv[cols], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
        assert s.solve() == ipm.IPM_OK
        out = s.get()
    assert kkt_check.rel_kkt(kkt_check.rt_ops(q), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-6


@pytest.mark.parametrize("storage", ["bf16", "fp8", "f32"])
def test_gap_layout_wide_gaps_and_ragged_columns(storage):
    """The reduced-precision column pass on 16-bit row gaps (cols_format = 1): V = 150000 voxel
    rows with one to three entries each over n = 3000 spots; some columns of R^T jump over more
    than 65535 rows (filler slots), every column ends in padding, some are empty.  Solved to
    the checker's tolerance, and against the same solve on int32 indices."""
    rng = np.random.default_rng(4)
    n, V = 3000, 150000
    k = rng.integers(1, 4, size=V)
    rows = [np.sort(rng.choice(n - 40, size=kk, replace=False)) for kk in k]
    # the last 40 columns: 20 hit only by rows 5, 70000 and 140000 (gaps of more than 65535
    # rows: filler slots), 20 by none (empty columns)
    for r in (5, 70000, 140000):
        rows[r] = np.concatenate([rows[r], np.arange(n - 40, n - 20)])
    k = np.array([len(a) for a in rows])
    ip = np.concatenate([[0], np.cumsum(k)]).astype(np.int64)
    ix = np.concatenate(rows).astype(np.int32)
    dv = rng.lognormal(0.0, 1.0, ix.size)
    w = rng.uniform(0.1, 10.0, V)
    d = (rng.random(V) < 0.3).astype(float)
    rowid = np.repeat(np.arange(V), k)
    c = -np.bincount(ix, weights=dv * (w * d)[rowid], minlength=n)
    a_rows = np.sort(rng.choice(np.flatnonzero(d == 0), size=500, replace=False)).astype(np.int32)
    p = dict(kind="rt", n=n, V=V, m=a_rows.size, D_indptr=ip, D_indices=ix, D_data=dv, w=w, d=d,
             h0=np.full(n, 1e-4), eps=1e-4, c=c, a_rows=a_rows, b=np.full(a_rows.size, 0.6), l=np.zeros(n),
             u=np.full(n, 5.0))
    col = np.sort(ix[np.argsort(ix, kind="stable")])
    rows_by_col = np.split(rowid[np.argsort(ix, kind="stable")], np.searchsorted(col, np.arange(1, n)))
    assert max(np.diff(r).max(initial=0) for r in rows_by_col) > 65535
    xs = []
    for cf in (1, 0):
        with ipm.Solver(tol_kkt=1e-6, storage=storage, cols_format=cf, max_cg=5000) as s:
            s.set_qp_rt(p)
            assert s.get_config()["cols_gap"] == (cf == 1)
            assert s.solve() == ipm.IPM_OK
            out = s.get()
        assert kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-6
        xs.append(out["x"])
    assert np.abs(xs[0] - xs[1]).max() <= 1e-3 * (1 + np.abs(xs[1]).max())


def test_double_float_refused_out_of_range():
    """Values beyond 2^90 would lose bits in a float32 pair: the handle keeps float64."""
    p = W.rt_qp(n=400, seed=15)
    big = dict(p)
    big["D_data"] = p["D_data"] * 2.0 ** 95
    big["w"] = p["w"] * 2.0 ** -190
    with ipm.Solver(tol_kkt=1e-8, op_arith="df32") as s:
        s.set_qp_rt(big)
        assert s.get_config()["op_arith"] == ipm.ARITH["f64"]
    with ipm.Solver(tol_kkt=1e-8, op_arith="df32") as s:
        s.set_qp_rt(p)
        assert s.get_config()["op_arith"] == ipm.ARITH["df32"]


def _mean_run(ip, ix):
    """Entries per run: a run starts at the first entry of a row or where the column is not one
    more than the previous entry's."""
    first = np.zeros(ix.size, bool)
    first[ip[:-1][np.diff(ip) > 0]] = True
    first[1:] |= ix[1:] != ix[:-1] + 1
    return ix.size / max(first.sum(), 1)


@pytest.mark.parametrize("n,density", [(2000, 0.02), (700, 0.005)])
@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_runs_auto_detection(n, density, storage):
    """AUTO takes runs for the reduced storages when they average at least 8 entries (banded
    dose rows at the RT density) and keeps CSR otherwise (short rows, scattered columns, or
    FP64 storage, where the CSR pass is as fast)."""
    p = W.rt_qp(n=n, seed=16, density=density)
    want = int(storage != "f64" and _mean_run(p["D_indptr"], p["D_indices"]) >= 8.0)
    with ipm.Solver(storage=storage) as s:
        s.set_qp_rt(p)
        assert s.get_config()["rows_runs"] == want
    rng = np.random.default_rng(3)
    n, m = 400, 300
    A = np.where(rng.random((m, n)) < 0.05, rng.normal(size=(m, n)), 0.0)
    with ipm.Solver(storage="bf16") as s:
        s.set_qp(n, m, rng.normal(size=n), np.abs(A).sum(1) + 1.0, np.zeros(n), np.ones(n), h0=np.ones(n),
                 A=_csr(A))
        assert s.get_config()["rows_runs"] == 0


def _csr(A):
    rows, cols = np.nonzero(A)
    ip = np.zeros(A.shape[0] + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=A.shape[0]), out=ip[1:])
    return ip, cols.astype(np.int32), A[rows, cols]
