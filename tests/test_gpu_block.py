"""The block-Jacobi preconditioner (32 x 32 diagonal blocks of H + A^T Theta A + Sigma, each
Cholesky-factored on the device every IPM iteration) against the oracle.

* Exactness of the blocks: when every row of the dose-like matrix lies inside one block of 32
  variables (and so does every constraint row), K itself is block diagonal, the
  preconditioner equals K, and PCG must meet a 1e-12 tolerance in one iteration (a wrong
  entry, a missed segment, a wrong weight or a transposed factor would not).  The last block
  is ragged (n not a multiple of 32).
* Directions and solves on RT-shaped, dense and quasi-Newton problems match the oracle as
  with the other preconditioners (PCG's answer does not depend on it, its iteration count
  does); a shared plan and the low-rank term update give the same bits.
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


def _blocky_rt(nb=40, tail=7, V=1500, seed=3):
    """RT-shaped QP whose every row of D holds a contiguous band inside one block of 32."""
    rng = np.random.default_rng(seed)
    n = 32 * nb + tail
    rows_i, rows_d = [], []
    for _ in range(V):
        b = rng.integers(0, nb + 1)
        lo, hi = 32 * b, min(32 * b + 32, n)
        ln = int(rng.integers(1, hi - lo + 1))
        c0 = int(rng.integers(lo, hi - ln + 1))
        rows_i.append(np.arange(c0, c0 + ln, dtype=np.int32))
        rows_d.append(rng.lognormal(0.0, 1.0, ln))
    ip = np.concatenate([[0], np.cumsum([len(a) for a in rows_i])]).astype(np.int64)
    ix = np.concatenate(rows_i)
    dv = np.concatenate(rows_d)
    w = rng.uniform(0.1, 10.0, V)
    d = (rng.random(V) < 0.3).astype(float)
    rowid = np.repeat(np.arange(V), np.diff(ip))
    c = -np.bincount(ix, weights=dv * (w * d)[rowid], minlength=n)
    a_rows = np.sort(rng.choice(np.flatnonzero(d == 0), size=V // 10, replace=False)).astype(np.int32)
    m = a_rows.size
    return dict(kind="rt", n=n, V=V, m=m, D_indptr=ip, D_indices=ix, D_data=dv, w=w, d=d, h0=np.full(n, 1e-4),
                eps=1e-4, c=c, a_rows=a_rows, b=np.full(m, 0.6), l=np.zeros(n), u=np.full(n, 5.0))


def test_blocks_are_exact_on_a_block_diagonal_problem():
    p = _blocky_rt()
    qp = O.from_rt(p)
    x, sl, y, zl, zu = W.random_iterate(qp.n, qp.m, qp.l, qp.u, 11, 1.0)
    it = O.Iterate(x, sl, y, zl, zu)
    with ipm.Solver(precond="block32", max_cg=50) as s:
        s.set_qp_rt(p)
        s.set_iterate(x, sl, y, zl, zu, 0.05)
        d = s.newton_direction(eta=1e-12)
        assert d["report"]["converged"] == 1 and d["report"]["iters"] == 1, d["report"]
        ref = O.newton_direction(qp, it, 0.05)
        assert np.abs(d["dx"] - ref.x).max() <= 1e-9 * np.abs(ref.x).max()
        # whole solve: one PCG iteration per Newton step (two where theta -> infinity makes a
        # block so ill-conditioned that one step's rounding misses the tolerance)
        assert s.solve() == ipm.IPM_OK
        assert all(t["pcg_iters"] <= 2 for t in s.trace())
        assert s.get()["info"]["precond"] == ipm.PRECOND["block32"]
    # the Jacobi diagonal alone needs many more on the same problem
    with ipm.Solver(precond="jacobi", max_cg=5000) as s:
        s.set_qp_rt(p)
        s.set_iterate(x, sl, y, zl, zu, 0.05)
        assert s.newton_direction(eta=1e-12)["report"]["iters"] > 5


@pytest.mark.parametrize("case", ["rt", "dense", "bfgs"])
def test_direction_and_solve_match_oracle(case):
    if case == "rt":
        p = W.rt_qp(n=1237, seed=3)
        qp, ops, load = O.from_rt(p), kkt_check.rt_ops(p), lambda s: s.set_qp_rt(p)
    elif case == "dense":
        p = W.dense_qp(n=300, m=700, seed=2)
        qp, ops = O.from_dense(p), kkt_check.dense_ops(p)
        load = lambda s: s.set_qp_dense(p["H"], p["c"], p["A"], p["b"], p["l"], p["u"])
    else:
        p = W.bfgs_qp(n=2000, k=10, m_ub=600, m_lb=200, density=0.01, seed=6, c_mode="target", ub_fac=1.1,
                      lb_fac=0.9)
        qp, ops, load = O.from_bfgs(p), kkt_check.bfgs_ops(p), lambda s: s.set_qp_bfgs(p)
    x, sl, y, zl, zu = W.random_iterate(qp.n, qp.m, qp.l, qp.u, 13, 1.0)
    it = O.Iterate(x, sl, y, zl, zu)
    ref = O.newton_direction(qp, it, 0.05)
    with ipm.Solver(precond="block32", max_cg=20000, tol_kkt=1e-7, stiff_max=1024) as s:
        load(s)
        s.set_iterate(x, sl, y, zl, zu, 0.05)
        d = s.newton_direction(eta=1e-12)
        assert d["report"]["converged"] == 1, d["report"]
        err = lambda a, b: np.abs(a - b).max() / (np.abs(b).max() + 1e-300)
        assert err(d["dx"], ref.x) <= 1e-7 and err(d["dzl"], ref.zl) <= 1e-7
        if qp.m:
            assert err(d["dy"], ref.y) <= 1e-7
        st = s.solve()
        out = s.get()
    assert st == ipm.IPM_OK, out["info"]
    assert kkt_check.rel_kkt(ops, out["x"], out["y"], out["zl"], out["zu"]) <= 1e-7
    sol, info = O.solve(qp, tol=1e-9)
    f, f0 = O.objective(qp, out["x"]), O.objective(qp, sol.x)
    assert abs(f - f0) / (1 + abs(f0)) <= 1e-6


def test_shared_plan_and_cost_update():
    """A slot sharing the plan forms its own fixed block part (from its own weights): the same
    bits as the plan; after ipm_update_costs both solve the new QP alike.  Reduced storage is
    refused with the block factors (as with the dense factor)."""
    for storage in ("bf16", "fp8", "f32"):
        with pytest.raises(ipm.IpmError):
            ipm.Solver(precond="block32", storage=storage)
    p = W.rt_qp(n=900, seed=7)
    with ipm.Solver(precond="block32", tol_kkt=1e-8) as plan, ipm.Solver(precond="block32", tol_kkt=1e-8) as slot:
        plan.set_qp_rt(p)
        slot.share_qp(plan)
        assert plan.solve() == ipm.IPM_OK and slot.solve() == ipm.IPM_OK
        assert np.array_equal(plan.get()["x"], slot.get()["x"])
        w2 = p["w"] * (1.0 + 0.01 * np.random.default_rng(1).normal(size=p["V"]))
        for s in (plan, slot):
            s.update_costs(f_w=w2)
            assert s.solve(warm=True) == ipm.IPM_OK
        assert np.array_equal(plan.get()["x"], slot.get()["x"])
        q = dict(p, w=w2)
        out = slot.get()
        assert kkt_check.rel_kkt(kkt_check.rt_ops(q), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-8


def test_unsorted_rows_refused():
    p = W.rt_qp(n=300, seed=8)
    ix = p["D_indices"].copy()
    r = int(np.argmax(np.diff(p["D_indptr"])))
    a, b = p["D_indptr"][r], p["D_indptr"][r + 1]
    ix[a:b] = ix[a:b][::-1].copy()
    q = dict(p, D_indices=ix, D_data=p["D_data"][::1].copy())
    q["D_data"][a:b] = p["D_data"][a:b][::-1]
    with ipm.Solver(precond="block32") as s:
        with pytest.raises(ipm.IpmError) as e:
            s.set_qp_rt(q)
        assert e.value.status == ipm.IPM_ERR_ARG
    with ipm.Solver(precond="jacobi_lr") as s:   # the other preconditioners take any order
        s.set_qp_rt(q)
        assert s.solve() == ipm.IPM_OK
