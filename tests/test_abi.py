"""The C-ABI library builds, loads and exports every symbol include/qcdgb.h declares (CPU only).

No compute call is made here: there is no GPU on the build host.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qcdgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(qcd_[A-Za-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1109_4279_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["qcd_create", "qcd_load_gauge", "qcd_build_clover", "qcd_apply_D", "qcd_solve",
              "qcd_solve_batch", "qcd_gradient", "qcd_autotune", "qcd_status_string", "qcd_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.qcd_status_string.restype = ctypes.c_char_p
    assert lib.qcd_status_string(0) == b"ok"
    assert b"even" in lib.qcd_status_string(-2)


def test_binding_names_match_header():
    from paper_1109_4279_gb300 import binding
    for n in _declared():
        if n in ("qcd_solver_defaults", "qcd_last_error"):
            continue
        assert hasattr(binding, n), n


def test_solver_params_layout_matches_header(lib):
    """qcd_solver_defaults (host only) fills the binding's structure: every
    field lands where the C layout puts it."""
    import ctypes
    from paper_1109_4279_gb300 import binding
    sp = binding.SolverParams()
    lib.qcd_solver_defaults(ctypes.byref(sp))
    assert (sp.tol, sp.nkv, sp.max_restarts, sp.precond, sp.ncy, sp.nmr) == (1e-10, 16, 100, 1, 4, 4)
    assert (sp.sap_prec, sp.outer_prec, sp.inner_tol, sp.solver, sp.ndefl) == (1, 0, 1e-5, 0, 4)
    assert (sp.cg_fallback, sp.cg_max_iter, sp.zero_guess, sp.residual_prec) == (0, 20000, 0, 4)
    assert ctypes.sizeof(binding.SolverParams) == 72  # LP64 layout of the C structure


def _params(dims, block, bc=(-1.0, 1.0, 1.0, 1.0)):
    from paper_1109_4279_gb300 import binding
    p = binding.Params()
    p.dims[:] = list(dims)
    p.block[:] = list(block)
    p.m0, p.csw = 0.0, 1.0
    p.bc[:] = list(bc)
    return p


@pytest.mark.parametrize("dims, block", [
    ((12, 4, 4, 4), (4, 2, 2, 2)),   # 3 blocks in direction 0: no chessboard colouring
    ((8, 6, 4, 4), (4, 3, 2, 2)),    # odd block extent: no even/odd split inside blocks
    ((8, 8, 4, 4), (4, 3, 2, 2)),    # block extent does not divide L
    ((32, 32, 16, 8), (16, 16, 8, 4)),  # Vb = 8192 > 4096, the largest block
    ((8, 8, 8, 0), (2, 2, 2, 2)),    # empty lattice
])
def test_create_rejects_bad_geometry_on_the_host(lib, dims, block):
    """Geometry is validated before any device call, so the checks run here."""
    import ctypes
    h = ctypes.c_void_p()
    st = lib.qcd_create(ctypes.byref(h), ctypes.byref(_params(dims, block)))
    assert st in (-2, -1) and not h.value  # QCD_ERR_GEOMETRY (QCD_ERR_ARG for a zero extent)


def test_create_rejects_bad_arguments_on_the_host(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.qcd_create(ctypes.byref(h), ctypes.byref(_params((8, 8, 8, 8), (4, 4, 2, 2), bc=(0.5, 1, 1, 1)))) == -1
    assert lib.qcd_create(None, ctypes.byref(_params((8, 8, 8, 8), (4, 4, 2, 2)))) == -1
    assert lib.qcd_create(ctypes.byref(h), None) == -1
    assert lib.qcd_solve(None, None, None, 1, None, None, None) == -1
