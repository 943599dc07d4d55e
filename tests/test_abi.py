"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/sapmg.h declares, the binding's struct layout matches, and the host-side
argument validation rejects bad input before any device work."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1202_2462_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libsapmg.so not built")
    return binding


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sapmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_setup", "dirac_apply", "sap_smooth", "mg_solve", "mg_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported():
    b = _lib()
    handle = ctypes.CDLL(b.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(handle, n)]
    assert not missing, missing


def test_params_layout_and_defaults():
    b = _lib()
    lib = b.lib()
    assert lib.mg_sizeof_params() == ctypes.sizeof(b.MgParams)
    p = b.mg_default_params()
    assert (p.n_levels, p.n_mr, p.nu_post, p.coarse_iters, p.fgmres_m) == (1, 4, 2, 12, 20)
    assert p.tol == 1e-10 and p.precision == b.MG_FP64 and list(p.agg2) == [2, 2, 2, 2]


@pytest.mark.parametrize("field,value", [
    ("dims", (8, 8, 12, 8)),       # 3 blocks of 4 in z: odd count
    ("dims", (8, 8, 8, 0)),
    ("n_levels", 7),
    ("coarse_iters", 40),
    ("tol", 0.0),
    ("precision", 9),
    ("setup2_iters", -1),
    ("setup2_iters", 1),           # set-up part 2 needs a coarse level (default: one level)
])
def test_setup_rejects_bad_params_on_host(field, value):
    b = _lib()
    p = b.mg_default_params()
    for mu in range(4):
        p.dims[mu] = 8
    if field == "dims":
        for mu in range(4):
            p.dims[mu] = value[mu]
    else:
        setattr(p, field, value)
    ctx = ctypes.c_void_p()
    # a non-null dummy pointer: validation happens before any device access
    code = b.lib().mg_setup(ctypes.c_void_p(16), 1.0, 0.0, ctypes.byref(p), ctypes.byref(ctx))
    assert code == b.MG_ERR_ARG
    assert ctx.value is None
    assert len(b.lib().mg_last_error()) > 0


def test_null_arguments_rejected():
    b = _lib()
    lib = b.lib()
    assert lib.dirac_apply(None, None, None, 0, 1) == b.MG_ERR_ARG
    assert lib.sap_smooth(None, None, None, 1, 0, 1) == b.MG_ERR_ARG
    assert lib.mg_solve(None, None, None, 1, None) == b.MG_ERR_ARG
    lib.mg_destroy(None)


def test_new_entry_points_reject_bad_arguments_on_host():
    """CGN, the set-up's host eigen-solvers: argument checks before any device work."""
    b = _lib()
    lib = b.lib()
    info = b.MgSolveInfo()
    assert lib.mg_cgn_solve(None, None, None, 1, b.MG_FP64, 1e-10, 10, ctypes.byref(info)) == b.MG_ERR_ARG
    assert lib.mg_harmonic_ritz(0, None, None, None) == b.MG_ERR_ARG
    assert lib.mg_eigh(0, None, None, None) == b.MG_ERR_ARG
    assert len(lib.mg_last_error()) > 0


def test_release_build_has_no_device_index_checks():
    """mg_debug_failures and mg_debug_check answer without a device in the
    release build: no checks compiled (-1), and the self-check refused."""
    b = _lib()
    if b.LIB_PATH.endswith("libsapmg_debug.so"):
        pytest.skip("the MG_DEBUG build is loaded")
    assert b.lib().mg_debug_failures() == -1
    assert b.lib().mg_debug_check(5, 3) == b.MG_ERR_STATE


def test_debug_build_exports_the_same_entry_points():
    from paper_1202_2462_gb300 import _build
    if not os.path.exists(_build.LIB_DEBUG):
        pytest.skip("libsapmg_debug.so not built (python -m paper_1202_2462_gb300._build --debug)")
    handle = ctypes.CDLL(_build.LIB_DEBUG)
    missing = [n for n in declared_functions() if not hasattr(handle, n)]
    assert not missing, missing
