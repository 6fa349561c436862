"""The C-ABI library builds, loads and exports every symbol of include/hofem.h (no GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "hofem.h")).read()
    return sorted(set(re.findall(r"\b(hofem_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_07758_gb300 import build as b
    b.build()
    import paper_1609_07758_gb300 as pkg
    return pkg.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "hofem_solve" in names and "hofem_plan" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    import paper_1609_07758_gb300.binding as bnd
    assert sorted(bnd.EXPORTED) == _declared()


def test_status_strings(lib):
    import paper_1609_07758_gb300 as pkg
    assert pkg.hofem_status_string(0) == "HOFEM_OK"
    assert pkg.hofem_status_string(1) == "HOFEM_ERR_INVALID_ARG"
    assert pkg.hofem_status_string(99) == "HOFEM_ERR_UNKNOWN"


@pytest.mark.parametrize("N,K,n,X,dtype,alpha", [
    (1, [8], 2, [1.0], 0, 0.0),                 # N must be 2 or 3
    (2, [8, 1], 2, [1.0, 1.0], 0, 0.0),         # K >= 2
    (2, [8, 8], 0, [1.0, 1.0], 0, 0.0),         # n >= 1
    (2, [8, 8], 17, [1.0, 1.0], 0, 0.0),        # n <= 16
    (2, [8, 8], 2, [1.0, -1.0], 0, 0.0),        # X > 0
    (2, [8, 8], 2, [1.0, 1.0], 0, -30.0),       # alpha > -pi^2 sum X^-2
])
def test_invalid_arguments_are_rejected_on_the_host(lib, N, K, n, X, dtype, alpha):
    out = ctypes.c_void_p()
    st = lib.hofem_plan(N, (ctypes.c_int * len(K))(*K), n, (ctypes.c_double * len(X))(*X), dtype, alpha,
                        ctypes.byref(out))
    assert st == 1 and not out.value


def test_per_axis_orders_are_checked_on_the_host(lib):
    out = ctypes.c_void_p()
    lib.hofem_plan_orders.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    Ks = (ctypes.c_int * 2)(8, 8)
    Xs = (ctypes.c_double * 2)(1.0, 1.0)
    for ns in ((2, 0), (17, 3)):
        assert lib.hofem_plan_orders(2, Ks, (ctypes.c_int * 2)(*ns), Xs, 0, 0.0, ctypes.byref(out)) == 1
    assert lib.hofem_plan_orders(2, Ks, None, Xs, 0, 0.0, ctypes.byref(out)) == 1


def test_unsupported_shapes_and_dtypes(lib):
    out = ctypes.c_void_p()
    Ks = (ctypes.c_int * 2)(16384, 8)        # K above 8192
    Xs = (ctypes.c_double * 2)(1.0, 1.0)
    assert lib.hofem_plan(2, Ks, 2, Xs, 0, 0.0, ctypes.byref(out)) == 2
    assert lib.hofem_plan(2, (ctypes.c_int * 2)(8, 8), 2, Xs, 7, 0.0, ctypes.byref(out)) == 2


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.hofem_solve(None, None, None, 1, None) == 1
    assert lib.hofem_apply(None, None, None, 1, None) == 1
    assert lib.hofem_set_refinement(None, 1, 0.0) == 1
    lib.hofem_destroy(None)


def test_slab_entry_points_check_arguments_on_the_host(lib):
    """The block sweep, block copy, slab residual and axpy entry points refuse bad arguments
    before touching a device (NULL plans, negative or inconsistent sizes, missing arrays)."""
    import paper_1609_07758_gb300  # noqa: F401  (argtypes)
    from paper_1609_07758_gb300 import binding
    binding.load_library()
    assert lib.hofem_sweep(None, 0, 0, None, None, 1, 1, 0, None) == 1
    assert lib.hofem_residual_slab(None, 0, 0, 1, None, None, None, None, None, 0, 1, None) == 1
    assert lib.hofem_copy_block(None, None, -1, 1, 1, 1, 1, 1, 1, None) == 1
    assert lib.hofem_copy_block(None, None, 1, 2, 4, 4, 4, 8, 8, None) == 1      # NULL arrays
    assert lib.hofem_copy_block(None, None, 1, 0, 4, 4, 4, 0, 0, None) == 0      # nothing to copy
    assert lib.hofem_axpy(None, 1.0, None, -1, None) == 1
    assert lib.hofem_axpy(None, 1.0, None, 0, None) == 0
    assert lib.hofem_axpy(None, 1.0, None, 5, None) == 1


def test_batch_and_tuner_host_checks(lib):
    out = ctypes.c_void_p()
    lib.hofem_batch_plan.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.hofem_batch_plan(0, None, 4, ctypes.byref(out)) == 1
    assert lib.hofem_batch_plan(1, None, 4, ctypes.byref(out)) == 1
    from paper_1609_07758_gb300.binding import hofem_problem
    bad = (hofem_problem * 2)()
    bad[0].N, bad[0].n, bad[0].nrhs = 2, 2, 1
    bad[1].N, bad[1].n, bad[1].nrhs = 4, 2, 1             # N must be 2 or 3
    assert lib.hofem_batch_plan(2, bad, 4, ctypes.byref(out)) == 1 and not out.value
    bad[1].N, bad[1].nrhs = 2, 0                           # nrhs >= 1
    assert lib.hofem_batch_plan(2, bad, 4, ctypes.byref(out)) == 1
    assert lib.hofem_batch_solve(None, None, None, None) == 1
    assert lib.hofem_batch_tune(None, None) == 1
    assert lib.hofem_batch_get_info(None, None) == 1
    assert lib.hofem_autotune(None, 1, None) == 1
    lib.hofem_batch_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_1609_07758_gb300.binding as bnd
    monkeypatch.setattr(bnd, "_lib", None)
    monkeypatch.setenv("HOFEM_LIBRARY", str(tmp_path / "nope.so"))
    with pytest.raises(bnd.HofemError):
        bnd.load_library()
