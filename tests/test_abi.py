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
    assert (sp.cg_fallback, sp.cg_max_iter) == (0, 20000)
