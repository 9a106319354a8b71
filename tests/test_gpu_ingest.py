"""ipm_set_qp's device-side R^T / A^T against the host transpose: identical results on every
problem family (bitwise equal solves), the long-column fallback, and the input checks."""
import numpy as np
import pytest

from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu


def _load(p, **opts):
    s = ipm.Solver(tol_kkt=1e-8, **opts)
    if p["kind"] == "rt":
        s.set_qp_rt(p)
    elif p["kind"] == "bfgs":
        s.set_qp_bfgs(p)
    else:
        s.set_qp_dense(p["H"], p["c"], p["A"], p["b"], p["l"], p["u"])
    return s


CASES = [
    ("rt_2311", lambda: W.rt_qp(n=2311, seed=41)),
    ("dense_120x260", lambda: W.dense_qp(n=120, m=260, seed=42)),
    ("bfgs_vmat_like", lambda: W.bfgs_qp(n=700, k=5, m_ub=900, m_lb=300, density=0.02, seed=43)),
    ("rt_long_columns", lambda: W.rt_qp(n=64, V=20000, density=0.3, seed=44, n_organ=300)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_device_ingest_equals_host(name, make):
    p = make()
    xs = []
    for host in (0, 1):
        with _load(p, ingest_host=host, precond="jacobi_lr") as s:
            assert s.solve() == ipm.IPM_OK
            out = s.get()
            xs.append((out["x"], out["info"]["ipm_iters"], out["info"]["cg_iters"]))
    assert np.array_equal(xs[0][0], xs[1][0]) and xs[0][1:] == xs[1][1:]


@pytest.mark.parametrize("host", [0, 1])
def test_ingest_rejects_bad_entries(host):
    p = W.rt_qp(n=300, seed=45)
    bad_idx = p["D_indices"].copy()
    bad_idx[len(bad_idx) // 2] = p["n"]
    bad_val = p["D_data"].copy()
    bad_val[7] = np.nan
    for idx, val, msg in ((bad_idx, p["D_data"], "column index"), (p["D_indices"], bad_val, "not finite")):
        s = ipm.Solver(ingest_host=host)
        with pytest.raises(ipm.IpmError) as e:
            s.set_qp(p["n"], p["m"], p["c"], p["b"], p["l"], p["u"], h0=p["h0"],
                     F=(p["D_indptr"], idx, val), f_w=p["w"], a_rows=p["a_rows"])
        assert e.value.status == ipm.IPM_ERR_ARG and msg in str(e.value)
        # the handle stays usable
        s.set_qp_rt(p)
        assert s.solve() == ipm.IPM_OK
        s.close()
