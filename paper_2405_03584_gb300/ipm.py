"""Python binding of the sm_103a interior point library (``include/ipm.h``), via ctypes.

Argument marshalling only: every step of the solve runs in the CUDA library.  Importing this
module does not load the library; the first use does, and raises if ``_lib/libipm.so`` is
missing (build it with ``paper_2405_03584_gb300.build.build()``).  There is no CPU fallback.

Arrays may be numpy arrays (host memory) or CUDA tensors (device memory, anything with
``data_ptr()`` and ``is_cuda``); all arrays of one call must live in the same memory space.
Streams default to PyTorch's current stream when PyTorch with CUDA is importable.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libipm.so")

IPM_OK, IPM_ERR_ARG, IPM_ERR_OOM, IPM_MAX_ITER, IPM_CG_STALL, IPM_NUMERICAL, \
    IPM_INFEASIBLE_SUSPECTED, IPM_ERR_TIMEOUT, IPM_ERR_CUDA, IPM_ERR_STATE, IPM_ERR_TOO_LARGE, IPM_BUSY = range(12)
STATIC_SCRATCH_ROWS = 262144
MEM_HOST, MEM_DEVICE = 0, 1
PRECOND = {"jacobi": 0, "jacobi_lr": 1, "dense": 2, "auto": 3, "block32": 4}
STORAGE = {"f64": 0, "f32": 1, "bf16": 2, "fp8": 3, "fp8_e4m3": 3}
ARITH = {"f64": 0, "df32": 1, "mixed": 2}
ROWS_FORMAT = {"auto": 0, "csr": 1, "runs": 2}
COLD, WARM = 0, 1

EXPORTS = ["ipm_default_options", "ipm_create", "ipm_set_qp", "ipm_solve", "ipm_get_xyz", "ipm_destroy",
           "ipm_status_str", "ipm_last_error", "ipm_set_iterate", "ipm_residuals", "ipm_apply_kkt",
           "ipm_precond_diag", "ipm_newton_direction", "ipm_step_lengths", "ipm_profile_operator",
           "ipm_get_trace", "ipm_apply_operator_static", "ipm_solve_async", "ipm_solve_wait", "ipm_solve_query",
           "ipm_batch_create", "ipm_batch_solve", "ipm_batch_destroy", "ipm_update_costs", "ipm_share_qp",
           "ipm_device_bytes", "ipm_set_lowrank", "ipm_abi_sizes", "ipm_get_sizes", "ipm_autotune_reset",
           "ipm_get_info"]
TRACE_COLS = ("iter", "mu", "rel_kkt", "primal", "dual", "gap", "alpha_p", "alpha_d", "pcg_iters", "pcg_converged",
              "stiff_rows", "pcg_rel_residual", "eta", "refine_passes")


class Options(C.Structure):
    _fields_ = [("tol_kkt", C.c_double), ("tau", C.c_double), ("max_ipm", C.c_int), ("max_cg", C.c_int),
                ("cg_eta_max", C.c_double), ("cg_eta_min", C.c_double), ("cg_eta_factor", C.c_double),
                ("precond", C.c_int), ("stiff_gamma", C.c_double), ("stiff_max", C.c_int),
                ("dense_max_n", C.c_int), ("timeout_ms", C.c_double), ("mem_budget", C.c_double),
                ("equal_steps", C.c_int), ("autotune", C.c_int), ("use_graphs", C.c_int),
                ("storage", C.c_int), ("refine_max", C.c_int), ("refine_eta", C.c_double),
                ("lanes_rows", C.c_int), ("lanes_cols", C.c_int), ("warm_rho", C.c_double),
                ("u_cap", C.c_int), ("ingest_host", C.c_int), ("system", C.c_int),
                ("lanes_at", C.c_int), ("op_arith", C.c_int), ("rows_format", C.c_int),
                ("rows_stage", C.c_int), ("wait_limit_ms", C.c_double), ("wait_test", C.c_int),
                ("cols_format", C.c_int), ("refine_mode", C.c_int)]


class QP(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("mem", C.c_int),
                ("c", C.c_void_p), ("b", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p),
                ("h0", C.c_void_p), ("H_dense", C.c_void_p), ("f_rows", C.c_int64),
                ("F_indptr", C.c_void_p), ("F_indices", C.c_void_p), ("F_data", C.c_void_p), ("f_w", C.c_void_p),
                ("a_rows", C.c_void_p), ("A_indptr", C.c_void_p), ("A_indices", C.c_void_p), ("A_data", C.c_void_p),
                ("u_cols", C.c_int64), ("U", C.c_void_p), ("u_w", C.c_void_p), ("bl", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("ipm_iters", C.c_int), ("cg_iters", C.c_int64), ("max_cg_step", C.c_int),
                ("max_stiff_rows", C.c_int), ("precond", C.c_int), ("rel_kkt", C.c_double),
                ("primal_res", C.c_double), ("dual_res", C.c_double), ("gap_res", C.c_double),
                ("primal_obj", C.c_double), ("dual_obj", C.c_double), ("mu", C.c_double), ("solve_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("lanes_rows", C.c_int), ("lanes_cols", C.c_int),
                ("refine_passes", C.c_int64), ("fallback_steps", C.c_int64), ("op_arith", C.c_int),
                ("rows_runs", C.c_int), ("cols_gap", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CgReport(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("stiff_rows", C.c_int),
                ("rel_res", C.c_double), ("eta", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Loads the library (once) and declares the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libipm.so not found at %s; build it with paper_2405_03584_gb300.build.build()" % path)
    L = C.CDLL(path)
    P, I, D, V = C.c_void_p, C.c_int, C.c_double, None
    sig = {
        "ipm_default_options": (V, [C.POINTER(Options)]),
        "ipm_create": (I, [C.POINTER(Options), C.POINTER(P)]),
        "ipm_set_qp": (I, [P, C.POINTER(QP), P]),
        "ipm_solve": (I, [P, P, I]),
        "ipm_get_xyz": (I, [P, P, P, P, P, P, C.POINTER(Info), I, P]),
        "ipm_destroy": (I, [P]),
        "ipm_status_str": (C.c_char_p, [I]),
        "ipm_last_error": (C.c_char_p, [P]),
        "ipm_set_iterate": (I, [P, P, P, P, P, P, D, I, P]),
        "ipm_residuals": (I, [P, P, P, P, P, P, P, I, P]),
        "ipm_apply_kkt": (I, [P, P, P, I, P]),
        "ipm_precond_diag": (I, [P, P, I, P]),
        "ipm_newton_direction": (I, [P, D, P, P, P, P, P, C.POINTER(CgReport), I, P]),
        "ipm_step_lengths": (I, [P, P, P, P, P, P, D, C.POINTER(C.c_double), C.POINTER(C.c_double), I, P]),
        "ipm_profile_operator": (I, [P, I] + [C.POINTER(C.c_double)] * 6),
        "ipm_get_trace": (I, [P, P, I]),
        "ipm_solve_async": (I, [P, P, I]),
        "ipm_solve_wait": (I, [P, C.POINTER(Info)]),
        "ipm_solve_query": (I, [P]),
        "ipm_batch_create": (I, [C.POINTER(P), I, I, C.POINTER(P)]),
        "ipm_batch_solve": (I, [P, P, C.POINTER(C.c_int)]),
        "ipm_batch_destroy": (I, [P]),
        "ipm_update_costs": (I, [P, P, P, I, P]),
        "ipm_share_qp": (I, [P, P, P]),
        "ipm_device_bytes": (I, [P, P, P, P]),
        "ipm_set_lowrank": (I, [P, C.c_int64, P, P, I, P]),
        "ipm_abi_sizes": (I, [P, P, P, P]),
        "ipm_get_sizes": (I, [P, P, P, P]),
        "ipm_autotune_reset": (I, []),
        "ipm_get_info": (I, [P, C.POINTER(Info)]),
        "ipm_apply_operator_static": (I, [C.c_int64, C.c_int64] + [P] * 10 + [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class IpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (load().ipm_status_str(status).decode(), status, msg))
        self.status = status


def _is_dev(a):
    return a is not None and hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


class _Marshal:
    """Keeps converted host arrays alive for the duration of one call."""

    def __init__(self, mem):
        self.mem = mem
        self.keep = []

    def ptr(self, a, dtype):
        if a is None:
            return None
        if self.mem == MEM_DEVICE:
            if not _is_dev(a):
                raise TypeError("mixed host and device arrays in one call")
            import torch
            want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
            if a.dtype != want or not a.is_contiguous():
                a = a.to(want).contiguous()
            self.keep.append(a)
            return a.data_ptr()
        arr = np.ascontiguousarray(np.asarray(a), dtype=dtype)
        self.keep.append(arr)
        return arr.ctypes.data


def _default_stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def autotune_reset():
    """Forgets the autotuner's per-matrix choices of this process (ipm_autotune_reset)."""
    return load().ipm_autotune_reset()


def default_options() -> dict:
    o = Options()
    load().ipm_default_options(C.byref(o))
    return {k: getattr(o, k) for k, _ in Options._fields_}


class Solver:
    """One solver handle.  Options are the fields of ipm_options (precond may be a name)."""

    def __init__(self, **opts):
        L = load()
        o = Options()
        L.ipm_default_options(C.byref(o))
        for k, v in opts.items():
            if k == "precond" and isinstance(v, str):
                v = PRECOND[v]
            if k == "storage" and isinstance(v, str):
                v = STORAGE[v]
            if k == "system" and isinstance(v, str):
                v = {"condensed": 0, "augmented": 1}[v]
            if k == "op_arith" and isinstance(v, str):
                v = ARITH[v]
            if k == "rows_format" and isinstance(v, str):
                v = ROWS_FORMAT[v]
            if not hasattr(o, k):
                raise TypeError("unknown option %s" % k)
            setattr(o, k, v)
        h = C.c_void_p()
        rc = L.ipm_create(C.byref(o), C.byref(h))
        if rc != IPM_OK:
            raise IpmError(rc, "ipm_create")
        self._h = h
        self.opts = o
        self.n = self.m = self.m_rows = 0

    # ---------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            load().ipm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, what, ok=(IPM_OK,)):
        if rc not in ok:
            raise IpmError(rc, "%s: %s" % (what, load().ipm_last_error(self._h).decode()))
        return rc

    # ---------------------------------------------------------------- problem
    def set_qp(self, n, m, c, b=None, l=None, u=None, h0=None, H_dense=None, F=None, f_w=None,
               a_rows=None, A=None, U=None, u_w=None, bl=None, stream=None):
        """F and A are CSR triplets (indptr int64, indices int32, data float64); U is n x k
        (row-major) with weights u_w: the low-rank Hessian term U diag(u_w) U^T.  bl gives
        two-sided rows bl <= A x <= b (-inf: no lower side; b may then hold +inf); get()
        then returns per row the signed multiplier y_upper - y_lower."""
        arrays = [c, b, l, u, h0, H_dense, f_w, a_rows, U, u_w, bl] + (list(F) if F else []) + (list(A) if A else [])
        mem = MEM_DEVICE if any(_is_dev(a) for a in arrays if a is not None) else MEM_HOST
        mk = _Marshal(mem)
        q = QP()
        q.n, q.m, q.mem = int(n), int(m), mem
        q.c = mk.ptr(c, np.float64)
        q.b = mk.ptr(b, np.float64) if m else None
        q.l = mk.ptr(l, np.float64)
        q.u = mk.ptr(u, np.float64)
        q.h0 = mk.ptr(h0, np.float64)
        q.H_dense = mk.ptr(H_dense, np.float64)
        if F is not None:
            ip, ix, dv = F
            q.f_rows = int(len(ip) - 1)
            q.F_indptr, q.F_indices, q.F_data = mk.ptr(ip, np.int64), mk.ptr(ix, np.int32), mk.ptr(dv, np.float64)
            q.f_w = mk.ptr(f_w, np.float64)
        if a_rows is not None and m:
            q.a_rows = mk.ptr(a_rows, np.int32)
        if A is not None and m:
            ip, ix, dv = A
            q.A_indptr, q.A_indices, q.A_data = mk.ptr(ip, np.int64), mk.ptr(ix, np.int32), mk.ptr(dv, np.float64)
        if U is not None:
            q.u_cols = int(U.shape[1]) if hasattr(U, "shape") else int(len(u_w))
            q.U, q.u_w = mk.ptr(U, np.float64), mk.ptr(u_w, np.float64)
        if bl is not None and m:
            q.bl = mk.ptr(bl, np.float64)
        self._check(load().ipm_set_qp(self._h, C.byref(q), _default_stream(stream)), "ipm_set_qp")
        self.n, self.m = int(n), int(m)
        self.m_rows = self.sizes()["m_rows"]
        return self

    def sizes(self):
        """dict(n, m, m_rows): m_rows counts the stored rows (two-sided rows stacked as [A; -A])."""
        n, m, mr = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(load().ipm_get_sizes(self._h, C.byref(n), C.byref(m), C.byref(mr)), "ipm_get_sizes")
        return dict(n=n.value, m=m.value, m_rows=mr.value)

    def set_qp_dense(self, H, c, A, b, l=None, u=None, bl=None, stream=None):
        """Dense QP: H as a dense symmetric block, A passed as CSR of its non-zeros (bl: lower
        sides of two-sided rows, as in set_qp)."""
        A = np.asarray(A, dtype=np.float64).reshape(-1, len(c))
        m, n = A.shape
        rows, cols = np.nonzero(A)
        indptr = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(np.bincount(rows, minlength=m), out=indptr[1:])
        Acsr = (indptr, cols.astype(np.int32), A[rows, cols]) if m else None
        return self.set_qp(n, m, c, b if m else None, l, u, H_dense=np.asarray(H, dtype=np.float64),
                           A=Acsr, bl=bl, stream=stream)

    def set_qp_rt(self, p, stream=None):
        """RT-shaped QP from ``workloads.rt_qp``: H = D^T diag(w) D + diag(h0), A = D[a_rows]
        (two-sided rows when p has "bl", as ``workloads.rt_two_sided`` gives)."""
        return self.set_qp(p["n"], p["m"], p["c"], p["b"], p["l"], p["u"], h0=p["h0"],
                           F=(p["D_indptr"], p["D_indices"], p["D_data"]), f_w=p["w"],
                           a_rows=p["a_rows"] if p["m"] else None, bl=p.get("bl"), stream=stream)

    def set_qp_bfgs(self, p, stream=None):
        """QP with a quasi-Newton Hessian from ``workloads.bfgs_qp``: H = diag(h0) + U diag(w) U^T,
        constraints (if any) as a CSR matrix A."""
        A = (p["A_indptr"], p["A_indices"], p["A_data"]) if p["m"] else None
        return self.set_qp(p["n"], p["m"], p["c"], p["b"] if p["m"] else None, p["l"], p["u"], h0=p["h0"],
                           A=A, U=p["U"], u_w=p["uw"], stream=stream)

    def set_lowrank(self, U=None, u_w=None, stream=None):
        """Replaces the low-rank Hessian term (U: n x k row-major, u_w: k); None drops it."""
        mk = _Marshal(MEM_HOST)
        k = 0 if U is None else int(np.asarray(U).shape[1])
        self._check(load().ipm_set_lowrank(self._h, k, mk.ptr(U, np.float64) if k else None,
                                           mk.ptr(u_w, np.float64) if k else None, MEM_HOST,
                                           _default_stream(stream)), "ipm_set_lowrank")

    def update_costs(self, f_w=None, c=None, stream=None):
        """New factor weights and/or linear cost for the loaded QP (matrices unchanged)."""
        mk = _Marshal(MEM_HOST)
        self._check(load().ipm_update_costs(self._h, mk.ptr(f_w, np.float64), mk.ptr(c, np.float64), MEM_HOST,
                                            _default_stream(stream)), "ipm_update_costs")

    def share_qp(self, src, stream=None):
        """Loads the QP of Solver ``src`` without copying its matrices (own state only)."""
        self._check(load().ipm_share_qp(self._h, src._h, _default_stream(stream)), "ipm_share_qp")
        self.n, self.m, self.m_rows = src.n, src.m, src.m_rows
        return self

    def device_bytes(self):
        """dict(matrix, state, matrix_refs): device bytes of the matrix store and of this handle's state."""
        mb, sb, refs = C.c_int64(), C.c_int64(), C.c_int()
        self._check(load().ipm_device_bytes(self._h, C.byref(mb), C.byref(sb), C.byref(refs)), "ipm_device_bytes")
        return dict(matrix=mb.value, state=sb.value, matrix_refs=refs.value)

    # ---------------------------------------------------------------- solve
    def solve(self, warm=False, stream=None):
        """Runs the IPM; returns the status code (IPM_OK on convergence)."""
        rc = load().ipm_solve(self._h, _default_stream(stream), WARM if warm else COLD)
        return self._check(rc, "ipm_solve", ok=(IPM_OK, IPM_MAX_ITER, IPM_CG_STALL, IPM_NUMERICAL,
                                                IPM_INFEASIBLE_SUSPECTED))

    def solve_async(self, warm=False, stream=None):
        """Queues the whole solve (one graph launch) and returns at once."""
        self._check(load().ipm_solve_async(self._h, _default_stream(stream), WARM if warm else COLD), "ipm_solve_async")

    def wait(self):
        """Waits for solve_async; returns the status."""
        info = Info()
        rc = load().ipm_solve_wait(self._h, C.byref(info))
        return self._check(rc, "ipm_solve_wait", ok=(IPM_OK, IPM_MAX_ITER, IPM_CG_STALL, IPM_NUMERICAL,
                                                     IPM_INFEASIBLE_SUSPECTED))

    def done(self):
        """True once the solve started by solve_async has finished (non-blocking)."""
        rc = load().ipm_solve_query(self._h)
        if rc not in (IPM_OK, IPM_BUSY):
            self._check(rc, "ipm_solve_query")
        return rc == IPM_OK

    def info(self):
        """ipm_info: the last solve's results and the operator configuration of the loaded QP."""
        info = Info()
        self._check(load().ipm_get_info(self._h, C.byref(info)), "ipm_get_info")
        return info.as_dict()

    def get_config(self):
        """The operator configuration chosen at set_qp: op_arith, rows_runs, cols_gap, lanes."""
        i = self.info()
        return {k: i[k] for k in ("op_arith", "rows_runs", "cols_gap", "lanes_rows", "lanes_cols")}

    def get(self, stream=None, out=None):
        """Returns dict(x, y, zl, zu, s, info).  ``out`` may give preallocated device tensors."""
        n, m = self.n, self.m
        info = Info()
        if out is None:
            x, y, zl, zu, s = np.empty(n), np.empty(m), np.empty(n), np.empty(n), np.empty(m)
            mem = MEM_HOST
            ptr = lambda a: a.ctypes.data if a.size else None
        else:
            x, y, zl, zu, s = (out[k] for k in ("x", "y", "zl", "zu", "s"))
            mem = MEM_DEVICE
            ptr = lambda a: a.data_ptr() if a is not None and a.numel() else None
        self._check(load().ipm_get_xyz(self._h, ptr(x), ptr(y), ptr(zl), ptr(zu), ptr(s), C.byref(info), mem,
                                       _default_stream(stream)), "ipm_get_xyz")
        return dict(x=x, y=y, zl=zl, zu=zu, s=s, info=info.as_dict())

    # ---------------------------------------------------------------- single steps
    def set_iterate(self, x, s, y, zl, zu, mu, stream=None):
        mk = _Marshal(MEM_HOST)
        self._check(load().ipm_set_iterate(self._h, mk.ptr(x, np.float64), mk.ptr(s, np.float64) if self.m_rows else None,
                                           mk.ptr(y, np.float64) if self.m_rows else None, mk.ptr(zl, np.float64),
                                           mk.ptr(zu, np.float64), float(mu), MEM_HOST, _default_stream(stream)),
                    "ipm_set_iterate")

    def residuals(self, stream=None):
        n, m = self.n, self.m_rows
        rd, rp, rs, rl, ru, kkt = np.empty(n), np.empty(m), np.empty(m), np.empty(n), np.empty(n), np.empty(4)
        p = lambda a: a.ctypes.data if a.size else None
        self._check(load().ipm_residuals(self._h, p(rd), p(rp), p(rs), p(rl), p(ru), p(kkt), MEM_HOST,
                                         _default_stream(stream)), "ipm_residuals")
        return dict(rd=rd, rp=rp, rs=rs, rl=rl, ru=ru, rel_kkt=kkt[0], primal=kkt[1], dual=kkt[2], gap=kkt[3])

    def apply_kkt(self, pvec, stream=None):
        pv = np.ascontiguousarray(pvec, dtype=np.float64)
        q = np.empty(self.n)
        self._check(load().ipm_apply_kkt(self._h, pv.ctypes.data, q.ctypes.data, MEM_HOST, _default_stream(stream)),
                    "ipm_apply_kkt")
        return q

    def precond_diag(self, stream=None):
        dg = np.empty(self.n)
        self._check(load().ipm_precond_diag(self._h, dg.ctypes.data, MEM_HOST, _default_stream(stream)),
                    "ipm_precond_diag")
        return dg

    def newton_direction(self, eta=0.0, stream=None):
        n, m = self.n, self.m_rows
        dx, ds, dy, dzl, dzu = np.empty(n), np.empty(m), np.empty(m), np.empty(n), np.empty(n)
        rep = CgReport()
        p = lambda a: a.ctypes.data if a.size else None
        self._check(load().ipm_newton_direction(self._h, float(eta), p(dx), p(ds), p(dy), p(dzl), p(dzu),
                                                C.byref(rep), MEM_HOST, _default_stream(stream)),
                    "ipm_newton_direction")
        return dict(dx=dx, ds=ds, dy=dy, dzl=dzl, dzu=dzu, report=rep.as_dict())

    def trace(self):
        """Per-IPM-iteration trace of the last solve as a list of dicts (keys TRACE_COLS)."""
        L = load()
        rows = L.ipm_get_trace(self._h, None, 0)
        buf = np.empty((max(rows, 1), len(TRACE_COLS)))
        L.ipm_get_trace(self._h, buf.ctypes.data, rows)
        return [dict(zip(TRACE_COLS, r)) for r in buf[:rows]]

    def profile_operator(self, reps=20):
        """Mean ms per launch and algorithmic bytes / flops of the two PCG operator kernels."""
        v = [C.c_double() for _ in range(6)]
        self._check(load().ipm_profile_operator(self._h, int(reps), *[C.byref(x) for x in v]), "ipm_profile_operator")
        keys = ("ms_rows", "ms_cols", "bytes_rows", "bytes_cols", "flops_rows", "flops_cols")
        return {k: x.value for k, x in zip(keys, v)}

    def step_lengths(self, dx, ds, dy, dzl, dzu, tau, stream=None):
        mk = _Marshal(MEM_HOST)
        ap, ad = C.c_double(), C.c_double()
        self._check(load().ipm_step_lengths(self._h, mk.ptr(dx, np.float64), mk.ptr(ds, np.float64) if self.m_rows else None,
                                            mk.ptr(dy, np.float64) if self.m_rows else None, mk.ptr(dzl, np.float64),
                                            mk.ptr(dzu, np.float64), float(tau), C.byref(ap), C.byref(ad), MEM_HOST,
                                            _default_stream(stream)), "ipm_step_lengths")
        return ap.value, ad.value


class Batch:
    """Many solver handles solved by one CUDA graph launch (one graph branch per handle)."""

    def __init__(self, solvers):
        L = load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        b = C.c_void_p()
        rc = L.ipm_batch_create(arr, len(self.solvers), COLD, C.byref(b))
        if rc != IPM_OK:
            raise IpmError(rc, "ipm_batch_create: %s" % L.ipm_last_error(self.solvers[0]._h).decode())
        self._b = b

    def solve(self, stream=None):
        """Runs every solve; returns the list of statuses."""
        st = (C.c_int * len(self.solvers))()
        rc = load().ipm_batch_solve(self._b, _default_stream(stream), st)
        if rc in (IPM_ERR_ARG, IPM_ERR_CUDA, IPM_ERR_STATE):
            raise IpmError(rc, "ipm_batch_solve")
        return list(st)

    def close(self):
        if getattr(self, "_b", None):
            load().ipm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
