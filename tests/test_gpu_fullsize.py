"""Parity at the benchmark's full size (RT-shaped QP, V = 200000, n = 50000, m = 20000) in the
launch configuration bench.py times (the same option set, ``presets.rt()``: tol_kkt = 1e-6,
JACOBI_LR, lanes per row picked by the autotuner).  The dense oracle cannot run
at this size, so the checks are the properties that hold at any size plus sampled outputs
evaluated one by one on the host:

* the returned point certifies with the independent checker (rel KKT <= 1e-6);
* the device's dual residual r_d equals the checker's, element by element;
* sampled entries of one operator apply q = (H + A^T Theta A + Sigma) p equal the entries
  evaluated from the definition;
* a mid-size instance of the same generator (n = 4000) matches the dense oracle's solution.
"""
import numpy as np
import pytest

from oracle import ipm as O
from oracle import kkt_check
from paper_2405_03584_gb300 import ipm, presets, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_2405_03584_gb300 import build
    build.build()
    p = W.rt_qp(n=50_000, seed=1)
    s = ipm.Solver(**presets.rt())
    s.set_qp_rt(p)
    st = s.solve()
    out = s.get()
    yield p, s, st, out
    s.close()


def test_full_size_certifies(full):
    p, s, st, out = full
    assert st == ipm.IPM_OK, out["info"]
    rk, det = kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"], detail=True)
    assert rk <= 1e-6, det
    assert abs(out["info"]["rel_kkt"] - rk) <= 1e-9 + 1e-6 * rk
    assert np.all(out["x"] > p["l"]) and np.all(out["x"] < p["u"]) and np.all(out["s"] > 0)


def test_full_size_residual_and_operator_samples(full):
    p, s, st, out = full
    r = s.residuals()
    rd = kkt_check.rt_residual_dual(p, out["x"], out["y"], out["zl"], out["zu"])
    scale = 1.0 + np.abs(rd).max()
    np.testing.assert_allclose(r["rd"], rd, rtol=1e-9, atol=1e-11 * scale * 1e3)
    rng = np.random.default_rng(4)
    pv = rng.normal(size=p["n"])
    q = s.apply_kkt(pv)
    cols = np.concatenate([[0, 1, p["n"] - 1], rng.choice(p["n"], 61, replace=False)])
    ref = kkt_check.rt_condensed_entries(p, out["x"], out["s"], out["y"], out["zl"], out["zu"], pv, cols)
    np.testing.assert_allclose(q[cols], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


@pytest.fixture(scope="module")
def mid():
    """The same generator at n = 4000 (V = 16000, m = 1600) and the oracle's solution."""
    p = W.rt_qp(n=4000, seed=1)
    qp = O.from_rt(p)
    ref, info = O.solve(qp, tol=1e-9)
    assert info.status == "optimal"
    return p, qp, ref


def test_mid_size_matches_oracle(mid):
    p, qp, ref = mid
    with ipm.Solver(tol_kkt=1e-7, precond="jacobi_lr") as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK
        out = s.get()
    f, f_ref = O.objective(qp, out["x"]), O.objective(qp, ref.x)
    assert abs(f - f_ref) / (1 + abs(f_ref)) <= 1e-6
    assert kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"]) <= 1e-7
    assert np.abs(out["x"] - ref.x).max() / (1 + np.abs(ref.x).max()) <= 1e-3


@pytest.mark.parametrize("storage,refine_mode", [("f64", 2), ("f32", 2), ("bf16", 2), ("fp8", 2), ("bf16", 0),
                                                 ("fp8", 1)])
def test_mid_size_error_per_storage(mid, storage, refine_mode):
    """Each operator storage in the benchmark's option set (refine_mode 2: the automatic choice
    of residual replacement or refinement passes; 0 and 1 force one), against the FP64 oracle:
    the error in x, in the objective and the relative KKT residual of the returned point (the
    precision configuration reports these per dtype).  Bars: rel. KKT <= 1e-6 and relative
    objective error <= 1e-6; the x error is printed (x* is unique, its distance follows the
    KKT residual through the conditioning of the problem)."""
    p, qp, ref = mid
    with ipm.Solver(**presets.rt(storage, refine_mode=refine_mode)) as s:
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK
        out = s.get()
    rk = kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"])
    f, f_ref = O.objective(qp, out["x"]), O.objective(qp, ref.x)
    ex = np.abs(out["x"] - ref.x).max() / np.abs(ref.x).max()
    e2 = np.linalg.norm(out["x"] - ref.x) / np.linalg.norm(ref.x)
    ef = abs(f - f_ref) / abs(f_ref)
    print("\nstorage-accuracy %s refine_mode %d: x_err_inf=%.3e x_err_2=%.3e obj_rel_err=%.3e rel_kkt=%.3e ipm=%d pcg=%d refine=%d"
          % (storage, refine_mode, ex, e2, ef, rk, out["info"]["ipm_iters"], out["info"]["cg_iters"], out["info"]["refine_passes"]))
    assert rk <= 1e-6
    assert ef <= 1e-6
