"""Shape and structure checks of the seeded synthetic generators."""
import numpy as np

from paper_2405_03584_gb300 import workloads as W


def test_dense_qp_structure():
    p = W.dense_qp(n=50, m=80, seed=0)
    np.testing.assert_allclose(p["Q"].T @ p["Q"], np.eye(50), atol=1e-12)
    assert p["lam"].min() >= 1e-3 and p["lam"].max() <= 1e2
    slack = p["b"] - p["A"] @ np.ones(50)
    assert slack.min() >= 0.1 and slack.max() <= 1.0
    q = W.dense_qp(n=50, m=80, seed=0)
    assert np.array_equal(p["H"], q["H"]) and np.array_equal(p["b"], q["b"])


def test_rt_qp_structure():
    p = W.rt_qp(n=2000, seed=3)
    V, n = p["V"], p["n"]
    ip, ix = p["D_indptr"], p["D_indices"]
    assert V == 4 * n and ip[-1] == ix.shape[0] and ix.dtype == np.int32
    for r in range(0, V, 997):
        row = ix[ip[r]:ip[r + 1]]
        assert np.all(np.diff(row) > 0) and row.min() >= 0 and row.max() < n
    dens = ip[-1] / (V * n)
    assert 0.004 < dens < 0.006
    assert np.all(p["D_data"] > 0)
    # constraint rows are non-target voxels; c = -D^T (w o d)
    assert np.all(p["d"][p["a_rows"]] == 0) and p["m"] == V // 10
    rows = np.repeat(np.arange(V), np.diff(ip))
    c = -np.bincount(ix, weights=p["D_data"] * (p["w"] * p["d"])[rows], minlength=n)
    np.testing.assert_allclose(p["c"], c)
    q = W.rt_qp(n=2000, seed=3)
    assert np.array_equal(p["D_data"], q["D_data"]) and np.array_equal(p["a_rows"], q["a_rows"])


def test_rt_batch_sizes_mix():
    sizes = W.rt_batch_sizes(64, seed=3)
    ns = np.array([s[0] for s in sizes])
    ds = np.array([s[1] for s in sizes])
    assert len(sizes) == 64 and ns.min() >= 2000 and ns.max() <= 40000
    assert ds.min() >= 0.002 and ds.max() <= 0.01


def test_rt_two_sided_structure():
    """Window rows: distinct from the organ rows and from each other, half targets, windows
    around the stated strictly feasible point, some rows lower-only, organ rows upper-only."""
    p = W.rt_qp(n=1200, seed=7)
    q = W.rt_two_sided(p, seed=2)
    m0 = p["m"]
    ar = q["a_rows"]
    assert q["m"] == ar.size and np.unique(ar).size == ar.size and np.array_equal(ar[:m0], p["a_rows"])
    win = ar[m0:]
    assert (p["d"][win] > 0).sum() == (p["d"][win] == 0).sum()
    assert np.all(np.isneginf(q["bl"][:m0])) and np.array_equal(q["b"][:m0], p["b"])
    assert np.all(np.isfinite(q["bl"][m0:])) and 0 < np.isinf(q["b"][m0:]).sum() < win.size
    # A x_f strictly inside every row's window, x_f inside the box
    xf = q["x_feasible"]
    rows = np.repeat(np.arange(p["V"]), np.diff(p["D_indptr"]))
    dose = np.bincount(rows, weights=p["D_data"] * xf[p["D_indices"]], minlength=p["V"])[ar]
    assert np.all(dose < q["b"]) and np.all(dose > q["bl"])
    assert np.all(xf > p["l"]) and np.all(xf < p["u"])
