"""CPU FP64 oracle for the GPU interior point method (test infrastructure only).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the CUDA library and its Python binding
never do, and the oracle never imports them.

* ``ipm``       -- plain primal-dual IPM with dense Cholesky Newton steps (Algorithm 1).
* ``kkt_check`` -- independent certificate checker: relative KKT residual of any point,
  evaluated with its own sparse matrix-vector products.
"""
