"""The allocation-free operator apply (ipm_apply_operator_static), for callers that cannot
allocate device memory, against the handle-based operator apply (ipm_apply_kkt) on the same
QP and iterate, and against the oracle's condensed matrix at that iterate: two calls in a
row, each checked element by element with the tolerance of the other operator tests (1e-10
relative).  Collected last on purpose (file name)."""
import numpy as np
import pytest

from oracle import ipm as O
from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu


def _csr_transpose(ip, ix, dv, ncols):
    """CSR of the transpose, rows in increasing order within each column (marshalling)."""
    nrows = ip.shape[0] - 1
    rows = np.repeat(np.arange(nrows, dtype=np.int32), np.diff(ip))
    order = np.argsort(ix, kind="stable")
    tp = np.zeros(ncols + 1, dtype=np.int64)
    np.cumsum(np.bincount(ix, minlength=ncols), out=tp[1:])
    return tp, rows[order], dv[order]


def test_static_scratch_operator_matches_apply_kkt():
    torch = pytest.importorskip("torch")
    from paper_2405_03584_gb300 import build
    build.build()
    L = ipm.load()
    p = W.rt_qp(n=700, seed=31)
    n, V, m = p["n"], p["V"], p["m"]
    x, s, y, zl, zu = W.random_iterate(n, m, p["l"], p["u"], 5, 1.0)
    solver = ipm.Solver(precond="jacobi")
    solver.set_qp_rt(p)
    solver.set_iterate(x, s, y, zl, zu, 0.3)
    # the operator's weights at this iterate: omega = w + theta on the constraint rows,
    # dg = h0 + z_l / (x - l) + z_u / (u - x)
    omega = p["w"].copy()
    omega[p["a_rows"]] += y / s
    dg = p["h0"] + zl / (x - p["l"]) + zu / (p["u"] - x)
    tp, ti, tv = _csr_transpose(p["D_indptr"], p["D_indices"], p["D_data"], n)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    f64, i64, i32 = torch.float64, torch.int64, torch.int32
    R = (dev(p["D_indptr"], i64), dev(p["D_indices"], i32), dev(p["D_data"], f64))
    RT = (dev(tp, i64), dev(ti, i32), dev(tv, f64))
    om, dgd = dev(omega, f64), dev(dg, f64)
    stream = torch.cuda.current_stream().cuda_stream
    qp = O.from_rt(p)
    it = O.Iterate(x, s, y, zl, zu)
    K, _, _, _ = O.condensed_system(qp, it, O.residuals(qp, it, 0.3))
    rng = np.random.default_rng(8)
    for call in range(2):
        pv = rng.normal(size=n)
        q_ref = solver.apply_kkt(pv)
        pd = dev(pv, f64)
        q = torch.full((n,), float("nan"), device="cuda", dtype=f64)
        rc = L.ipm_apply_operator_static(n, V, R[0].data_ptr(), R[1].data_ptr(), R[2].data_ptr(),
                                         RT[0].data_ptr(), RT[1].data_ptr(), RT[2].data_ptr(),
                                         om.data_ptr(), dgd.data_ptr(), pd.data_ptr(), q.data_ptr(), stream)
        assert rc == ipm.IPM_OK, (call, rc)
        torch.cuda.synchronize()
        qh = q.cpu().numpy()
        np.testing.assert_allclose(qh, q_ref, rtol=1e-10, atol=1e-12 * np.abs(q_ref).max(), err_msg="call %d" % call)
        kp = K @ pv
        np.testing.assert_allclose(qh, kp, rtol=1e-10, atol=1e-12 * np.abs(K).max() * np.abs(pv).max() * n,
                                   err_msg="oracle, call %d" % call)
    # more rows than the fixed scratch holds: refused before any work
    rc = L.ipm_apply_operator_static(n, ipm.STATIC_SCRATCH_ROWS + 1, R[0].data_ptr(), R[1].data_ptr(),
                                     R[2].data_ptr(), RT[0].data_ptr(), RT[1].data_ptr(), RT[2].data_ptr(),
                                     om.data_ptr(), dgd.data_ptr(), pd.data_ptr(), q.data_ptr(), stream)
    assert rc == ipm.IPM_ERR_TOO_LARGE
    solver.close()
