"""Every lane-group width of the templated row kernels, pinned to the oracle.

The row kernels over R (operator rows pass, residual rows pass), over R^T (operator column
pass, residual column pass) and over A^T (right-hand side with the Jacobi diagonal, Jacobi
diagonal) are instantiated for 4, 8, 16 and 32 lanes per row, and the autotuner or the
options pick one per matrix.  Here every width of each is run on one RT-shaped instance with
ragged rows (n = 1237: row lengths from a binomial, several blocks, no multiple of any
width) and compared element by element with the oracle at the same iterate:

* FP64 storage: residuals (1e-10 relative), one operator apply q = K p against the oracle's
  condensed matrix (1e-10), the Jacobi diagonal (1e-11) and one Newton direction at
  eta = 1e-12 (1e-7 relative, the bound cond(K) * eta gives);
* F32 / BF16 / FP8 storage: the refined Newton direction (FP32 PCG inside FP64 refinement)
  at eta = 1e-10 against the oracle's exact direction (1e-6 relative).

Each FP64-storage check runs for both operator arithmetics (float64, double-float) and both
formats of the rows pass (CSR, runs; double-float runs also staged through shared memory by
bulk copies); the reduced storages for every rows format, with the column pass on int32
indices (the default) and on 16-bit row gaps.
"""
import itertools

import numpy as np
import pytest

from oracle import ipm as O
from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu

WIDTHS = (4, 8, 16, 32)
PAIRS = list(itertools.product(WIDTHS, WIDTHS))
MU = 0.05


@pytest.fixture(scope="module")
def case():
    from paper_2405_03584_gb300 import build
    build.build()
    ipm.load()
    p = W.rt_qp(n=1237, seed=3)
    qp = O.from_rt(p)
    x, sl, y, zl, zu = W.random_iterate(qp.n, qp.m, qp.l, qp.u, 7, 1.0)
    it = O.Iterate(x, sl, y, zl, zu)
    res = O.residuals(qp, it, MU)
    K, _, _, _ = O.condensed_system(qp, it, res)
    ref_dir = O.newton_direction(qp, it, MU)
    lens = np.diff(p["D_indptr"])
    assert lens.min() != lens.max() and p["V"] % 32 and p["n"] % 32 and p["m"] % 32
    return p, qp, it, res, K, ref_dir


def _err(a, b):
    return np.abs(a - b).max() / (np.abs(b).max() + 1e-300)


VARIANTS = [("f64", "csr"), ("f64", "runs"), ("df32", "csr"), ("df32", "runs"), ("df32", "runs-staged"), ("mixed", "csr")]


def _fmt(fmt):
    """Options of a variant name: the rows format first ("csr", "runs"), then "-staged" (the
    pieces streamed through the shared-memory copy pipeline instead of read from global
    memory), "-colsgap" (the reduced-precision column pass on the 16-bit row-gap layout
    instead of int32 indices) or "-ru" (one PCG with residual replacement per Newton step
    instead of restarted refinement passes)."""
    return dict(rows_format=fmt.split("-")[0], rows_stage=1 if fmt.endswith("-staged") else 0,
                cols_format=1 if fmt.endswith("-colsgap") else 0, refine_mode=1 if fmt.endswith("-ru") else 0)


@pytest.mark.parametrize("arith,fmt", VARIANTS, ids=["%s-%s" % v for v in VARIANTS])
@pytest.mark.parametrize("lr,lc", PAIRS, ids=["rows%d-cols%d" % pc for pc in PAIRS])
def test_fp64_kernels_every_width(case, lr, lc, arith, fmt):
    p, qp, it, (rd, rp, rs, rl, ru), K, ref_dir = case
    la = lr   # the A^T kernels take every width across the sweep as well
    with ipm.Solver(precond="jacobi_lr", lanes_rows=lr, lanes_cols=lc, lanes_at=la, max_cg=20000,
                    op_arith=arith, **_fmt(fmt)) as s:
        s.set_qp_rt(p)
        s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, MU)
        r = s.residuals()
        np.testing.assert_allclose(r["rd"], rd, rtol=1e-10, atol=1e-11 * (1 + np.abs(rd).max()))
        np.testing.assert_allclose(r["rp"], rp, rtol=1e-10, atol=1e-11 * (1 + np.abs(rp).max()))
        rng = np.random.default_rng(lr * 100 + lc)
        pv = rng.normal(size=qp.n)
        q = s.apply_kkt(pv)
        np.testing.assert_allclose(q, K @ pv, rtol=1e-10, atol=1e-12 * np.abs(K).max() * np.abs(pv).max() * qp.n)
        np.testing.assert_allclose(s.precond_diag(), np.diag(K), rtol=1e-11)
        d = s.newton_direction(eta=1e-12)
        assert d["report"]["converged"] == 1, d["report"]
        info = s.get()["info"]
        assert info["op_arith"] == ipm.ARITH[arith] and info["rows_runs"] == fmt.startswith("runs")
        assert _err(d["dx"], ref_dir.x) <= 1e-7
        assert _err(d["dy"], ref_dir.y) <= 1e-7 and _err(d["ds"], ref_dir.s) <= 1e-7
        assert _err(d["dzl"], ref_dir.zl) <= 1e-7 and _err(d["dzu"], ref_dir.zu) <= 1e-7


@pytest.mark.parametrize("fmt", ["csr", "runs", "runs-staged", "runs-colsgap", "runs-ru"])
@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("lr,lc", PAIRS, ids=["rows%d-cols%d" % pc for pc in PAIRS])
def test_reduced_precision_kernels_every_width(case, storage, lr, lc, fmt):
    p, qp, it, _, _, ref_dir = case
    with ipm.Solver(precond="jacobi_lr", storage=storage, lanes_rows=lr, lanes_cols=lc, lanes_at=lc,
                    max_cg=5000, refine_max=30, **_fmt(fmt)) as s:
        s.set_qp_rt(p)
        s.set_iterate(it.x, it.s, it.y, it.zl, it.zu, MU)
        d = s.newton_direction(eta=1e-10)
        assert d["report"]["converged"] == 1, d["report"]
        assert _err(d["dx"], ref_dir.x) <= 1e-6
        assert _err(d["dy"], ref_dir.y) <= 1e-6
