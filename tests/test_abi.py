"""The C-ABI library builds, loads without a GPU and exports every function that
include/fmg.h declares; the Python binding carries the same names.  Host-side
argument validation is exercised where it needs no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fmg_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg

    return fmg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fmg_create", "fmg_solve", "fmg_solve_batch", "fmg_destroy", "fmg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_has_same_names(lib):
    from paper_1611_05677_gb300 import fmg

    for name in declared_functions():
        assert callable(getattr(fmg, name)), name
    assert set(fmg.EXPORTS) == set(declared_functions())


def test_default_params_and_validation(lib):
    from paper_1611_05677_gb300 import fmg

    p = fmg.fmg_default_params()
    assert (p.dim, p.coarse_cells, p.refinements, p.m_vcycles, p.nu_pre, p.nu_post, p.p_corrections) == (
        2, 4, 4, 2, 2, 2, 1)
    assert fmg.fmg_workspace_bytes(p) > 0
    for field, bad in (("dim", 4), ("coarse_cells", 3), ("coarse_cells", 16), ("refinements", -1),
                       ("f", 9), ("f_scale", -1.0), ("m_vcycles", 0), ("p_corrections", 0),
                       ("precision", 7), ("newton_maxit", 0), ("newton_tol", 0.0)):
        q = fmg.fmg_default_params()
        setattr(q, field, bad)
        with pytest.raises(fmg.FMGError) as ei:
            fmg.fmg_workspace_bytes(q)
        assert ei.value.status == fmg.FMG_ERR_INVALID
        assert fmg.fmg_last_error()


def test_coefficient_validation(lib):
    """The coefficient table is checked entry by entry (finite, > 0) and only with the
    red-black smoother; its size follows coarse_cells^dim rows of dim entries."""
    from paper_1611_05677_gb300 import fmg
    from paper_1611_05677_gb300 import workloads as W

    for dim, nc in ((2, 4), (3, 2)):
        coef = W.cell_coefficient(dim, nc)
        p = fmg.make_params(dim=dim, coarse_cells=nc, refinements=2, coefficient=coef)
        assert fmg.fmg_workspace_bytes(p) > 0
        for bad in (0.0, -1.0, float("nan"), float("inf")):
            c2 = coef.copy()
            c2[-1, -1] = bad
            q = fmg.make_params(dim=dim, coarse_cells=nc, refinements=2, coefficient=c2)
            with pytest.raises(fmg.FMGError) as ei:
                fmg.fmg_workspace_bytes(q)
            assert ei.value.status == fmg.FMG_ERR_INVALID
            assert "coefficient" in fmg.fmg_last_error()
        q = fmg.make_params(dim=dim, coarse_cells=nc, refinements=2, coefficient=coef, smoother="chebyshev")
        with pytest.raises(fmg.FMGError) as ei:
            fmg.fmg_workspace_bytes(q)
        assert ei.value.status == fmg.FMG_ERR_INVALID
        with pytest.raises(fmg.FMGError):
            fmg.make_params(dim=dim, coarse_cells=nc, refinements=2, coefficient=coef[:-1])


def test_null_arguments_are_rejected(lib):
    from paper_1611_05677_gb300 import fmg

    assert lib.fmg_destroy(None) == fmg.FMG_OK
    assert lib.fmg_solve(None, None, 1, None) == fmg.FMG_ERR_INVALID
    assert lib.fmg_levels(None) == -1
    assert lib.fmg_level_cells(None, 1) == -1
    out = ctypes.c_void_p()
    p = fmg.fmg_default_params()
    assert lib.fmg_create(ctypes.byref(p), None, 0, None, None, 0, ctypes.byref(out)) == fmg.FMG_ERR_INVALID
    assert not out.value
    # batches: a NULL context anywhere in the list is rejected before any context is touched
    two = (ctypes.c_void_p * 2)(None, None)
    assert lib.fmg_solve_batch(two, 2, None, None) == fmg.FMG_ERR_INVALID
    assert lib.fmg_solve_batch(None, 1, None, None) == fmg.FMG_ERR_INVALID
    batch = ctypes.c_void_p()
    assert lib.fmg_batch_create(two, 2, None, ctypes.byref(batch)) == fmg.FMG_ERR_INVALID
    for mode in (fmg.BATCH_AUTO, fmg.BATCH_PHASES, fmg.BATCH_BRANCHES, 7):
        assert lib.fmg_batch_create_mode(two, 2, None, mode, 0, ctypes.byref(batch)) == fmg.FMG_ERR_INVALID
    assert b"unknown batch mode" in lib.fmg_last_error(None)
    assert lib.fmg_batch_info(None, None, None, None) == fmg.FMG_ERR_INVALID
    assert lib.fmg_batch_destroy(None) == fmg.FMG_OK
    # the request server's calls reject NULL servers
    assert lib.fmg_server_submit(None, None, None, None, None) == fmg.FMG_ERR_INVALID
    assert lib.fmg_server_poll(None, None, 1) == 0
    assert lib.fmg_server_destroy(None) == fmg.FMG_OK


def test_workspace_grows_with_levels(lib):
    from paper_1611_05677_gb300 import fmg

    a = fmg.fmg_workspace_bytes(fmg.make_params(refinements=3))
    b = fmg.fmg_workspace_bytes(fmg.make_params(refinements=4))
    c = fmg.fmg_workspace_bytes(fmg.make_params(refinements=4, precision="mixed"))
    assert a < b < c
    # three FP64 nodal arrays per level at least
    assert b >= 3 * 8 * (65 ** 2 + 33 ** 2 + 17 ** 2 + 9 ** 2 + 5 ** 2)
