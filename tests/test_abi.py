"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/ipm.h declares, and its host-only calls behave (no compute calls here)."""
import ctypes as C
import os
import re

import pytest

from paper_2405_03584_gb300 import build, ipm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ipm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ipm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ipm.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(ipm.EXPORTS) <= set(names)


def test_default_options(lib):
    o = ipm.default_options()
    assert o["tol_kkt"] == 1e-6 and o["tau"] == 0.995 and o["max_ipm"] == 200
    assert o["precond"] == ipm.PRECOND["auto"] and o["stiff_max"] == 256


def test_status_strings(lib):
    for code in range(10):
        assert lib.ipm_status_str(code)
    assert lib.ipm_status_str(0) == b"ok"


def test_null_arguments_rejected(lib):
    assert lib.ipm_create(None, None) == ipm.IPM_ERR_ARG
    assert lib.ipm_destroy(None) == ipm.IPM_OK
    assert lib.ipm_set_qp(None, None, None) == ipm.IPM_ERR_ARG
    assert lib.ipm_solve(None, None, 0) == ipm.IPM_ERR_ARG
    bad = ipm.Options()
    lib.ipm_default_options(C.byref(bad))
    bad.tau = 1.5
    h = C.c_void_p()
    assert lib.ipm_create(C.byref(bad), C.byref(h)) == ipm.IPM_ERR_ARG


@pytest.mark.parametrize("field,value", [
    ("precond", 2), ("precond", 4), ("precond", 5), ("system", 1), ("stiff_max", 1025), ("lanes_rows", 12),
    ("lanes_at", 3), ("op_arith", 3), ("rows_format", 3), ("rows_stage", 2), ("wait_limit_ms", 0.0),
    ("dense_max_n", 4096),
    ("refine_eta", 1.0), ("refine_eta", -0.1), ("refine_mode", 3), ("warm_rho", 1.0), ("u_cap", 1 << 17), ("storage", 4)])
def test_invalid_option_combinations_rejected(lib, field, value):
    """ipm_create validates the options before touching the device: with BF16 storage the
    DENSE preconditioner and the doubly augmented system are refused, and so are values
    outside their documented ranges."""
    o = ipm.Options()
    lib.ipm_default_options(C.byref(o))
    o.storage = ipm.STORAGE["bf16"]
    setattr(o, field, value)
    h = C.c_void_p()
    assert lib.ipm_create(C.byref(o), C.byref(h)) == ipm.IPM_ERR_ARG
    assert not h.value


def test_static_operator_argument_checks(lib):
    """The allocation-free operator refuses bad arguments and sizes beyond its fixed scratch
    before any device work (the pointers below are never dereferenced)."""
    f = lib.ipm_apply_operator_static
    d = C.c_void_p(16)
    ok = [d] * 10          # R_indptr, R_indices, R_data, RT_indptr, RT_indices, RT_data, omega, dg, p, q
    assert f(0, 0, *ok, None) == ipm.IPM_ERR_ARG
    assert f(10, -1, *ok, None) == ipm.IPM_ERR_ARG
    # each pointer NULL in turn, at a small nR: refused before any launch
    for k in range(10):
        args = list(ok)
        args[k] = None
        assert f(10, 5, *args, None) == ipm.IPM_ERR_ARG, k
    # with nR = 0 the arrays of R and omega are not needed; those of R^T still are
    for k in range(10):
        args = list(ok)
        args[k] = None
        want = ipm.IPM_ERR_ARG if k in (3, 4, 5, 7, 8, 9) else None
        if want is not None:
            assert f(10, 0, *args, None) == want, k
    too_many = (1 << 18) + 1
    assert f(10, too_many, *ok, None) == ipm.IPM_ERR_TOO_LARGE
    # a NULL pointer is reported as such even beyond the size limit
    assert f(10, too_many, d, None, d, d, d, d, d, d, d, d, None) == ipm.IPM_ERR_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(ipm, "_lib", None)
    with pytest.raises(ImportError):
        ipm.load(str(tmp_path / "nope.so"))


def test_struct_layouts_match_the_library(lib):
    """The binding's ctypes structs have the sizes the library was compiled with."""
    sizes = [C.c_int64() for _ in range(4)]
    assert lib.ipm_abi_sizes(*[C.byref(v) for v in sizes]) == ipm.IPM_OK
    ours = [C.sizeof(ipm.Options), C.sizeof(ipm.QP), C.sizeof(ipm.Info), C.sizeof(ipm.CgReport)]
    assert [v.value for v in sizes] == ours
