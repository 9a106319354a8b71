"""The uneven batch (many RT-shaped QPs of different sizes, FP32 operator storage with FP64
refinement, one graph launch) against the CPU oracle on its smallest instances, and every
instance certified by the independent checker."""
import numpy as np
import pytest

from oracle import ipm as O
from oracle import kkt_check
from paper_2405_03584_gb300 import ipm, workloads as W

pytestmark = pytest.mark.gpu


def test_uneven_batch_matches_oracle():
    from paper_2405_03584_gb300 import build
    build.build()
    probs = W.rt_batch(12, seed=3, scale=0.05)          # n from about 100 to 2000
    solvers = []
    for p in probs:
        s = ipm.Solver(tol_kkt=1e-7, precond="jacobi_lr", storage="f32", autotune=1)
        s.set_qp_rt(p)
        solvers.append(s)
    b = ipm.Batch(solvers)
    st = b.solve()
    assert st == [ipm.IPM_OK] * len(probs)
    order = np.argsort([p["n"] for p in probs])
    for k, i in enumerate(order):
        p, out = probs[i], solvers[i].get()
        rk = kkt_check.rel_kkt(kkt_check.rt_ops(p), out["x"], out["y"], out["zl"], out["zu"])
        assert rk <= 1e-7 * 1.0001, (i, rk)
        if k < 6:                                       # oracle on the six smallest instances
            qp = O.from_rt(p)
            ref, info = O.solve(qp, tol=1e-8)
            assert info.status == "optimal"
            f, f_ref = O.objective(qp, out["x"]), O.objective(qp, ref.x)
            assert abs(f - f_ref) / (1 + abs(f_ref)) <= 1e-6
    b.close()
    for s in solvers:
        s.close()
