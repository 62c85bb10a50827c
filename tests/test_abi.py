"""The C-ABI library builds, loads on a machine without a GPU and exports
every entry point that include/wsi.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wsi_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("wsi_create_grid", "wsi_set_phases", "wsi_stokes_solve", "wsi_dlm_constrain", "wsi_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1901_07892_gb300 import wsi
    L = wsi.lib()
    for n in _declared():
        assert hasattr(L, n), n
    assert set(_declared()) <= set(wsi.EXPORTED)


def test_invalid_arguments_rejected_without_gpu_work():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1901_07892_gb300 import wsi
    L = wsi.lib()
    d = wsi.GridDesc(0, 4, 4, 1.0, 1.0, 1.0, (ctypes.c_double * 6)(*([-1.0] * 6)),
                     (ctypes.c_double * 3)(0, 0, -9.81), 2.0, 0.5, 0, 2, 2, 1, 2, 20)
    h = ctypes.c_void_p()
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.nx = 4
    d.bc[0] = 0.5  # not a wall sign
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    assert L.wsi_stokes_solve(None, None, None, 1.0, None, None) == wsi.ERR_INVALID_ARG
    d.bc[0] = -1.0
    d.reinit_iters = -1  # negative pseudo-time step count
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.reinit_iters = 0
    d.transport_form = 7  # neither formulation
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.transport_form = wsi.FORM_CONSISTENT
    d.mg_smoother = 3  # neither smoother
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.mg_smoother = wsi.SMOOTH_RBGS
    d.ls_limiter = 2  # neither limiter
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.ls_limiter = wsi.LIMIT_CUI
    d.open_top = 2  # neither closed nor open
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.open_top = 1
    d.bc[5] = 1.0  # an open top has zero tangential velocity: the lid's sign must be no-slip
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.bc[5] = -1.0
    d.visc_mg = 1  # the viscous V-cycle has no open-top rows
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    d.visc_mg = 0
    d.open_top = 0
    d.precision = 5
    assert L.wsi_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == wsi.ERR_INVALID_ARG
    assert L.wsi_reinit(None, None, 3) == wsi.ERR_INVALID_ARG
    assert L.wsi_step(None, 1e-3, None, None) == wsi.ERR_INVALID_ARG
