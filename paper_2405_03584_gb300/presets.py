"""Solver option sets under which the RT-shaped workload is benchmarked, shared by bench.py
and the full-size parity tests, so that the kernels the benchmark times are the kernels the
tests certify."""

# The RT-shaped QP (200000 x 50000 dose-like matrix, 20000 organ rows), FP64 storage.
RT_FP64 = dict(tol_kkt=1e-6, precond="jacobi_lr", autotune=1)


def rt(storage="f64", **extra):
    """Options of the RT benchmark for the given operator storage (reduced storages add FP64
    refinement of every Newton step)."""
    o = dict(RT_FP64)
    o["storage"] = storage
    o.update(extra)
    return o
