"""Plain FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
``oracle.c`` is compiled on its own by :func:`build` into ``liboracle.so`` and
reached through ctypes; ``dense.py`` is an independent numpy assembler of the
same operator used to pin the C oracle.

Field conventions (all numpy complex128, C order, lexicographic sites with
x0 = time slowest): gauge ``(V, 4, 3, 3)``, spinor ``(V, 4, 3)``, clover
``(V, 12, 12)`` with row index ``spin * 3 + colour`` and the ``4 + m0`` mass
term on the diagonal.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc/OpenMP into ``liboracle.so`` (in-tree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def bind(cdll):
    """Declare the argument and result types of the oracle's C entry points on
    a loaded library (the built liboracle.so, or a variant a test compiled)."""
    d, i, l = ctypes.c_void_p, ctypes.c_int, ctypes.c_long
    for name, args in {
        "oracle_clover": [d, d, ctypes.c_double, ctypes.c_double, d],
        "oracle_apply_D": [d, d, d, d, d, d, i],
        "oracle_dD_apply": [d, d, d, d, ctypes.c_double, d, d],
        "oracle_sap": [d, d, d, d, d, i, i, i, i, d, d, d],
        "oracle_block_mr": [d, d, d, d, d, l, i, i, d, d],
        "oracle_block_sites": [d, d, l, d],
        "oracle_fgcr": [d, d, d, d, d, d, i, i, ctypes.c_double, i, d, i, i, i, i, d, d],
        "oracle_num_threads": [],
    }.items():
        fn = getattr(cdll, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return cdll


def lib():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(build()))
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _dims(L):
    return np.ascontiguousarray(np.asarray(L, dtype=np.int32))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _bc(bc):
    return np.ascontiguousarray(np.asarray(bc, dtype=np.float64))


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"{what} failed with status {st}")


def num_threads() -> int:
    return lib().oracle_num_threads()


def clover(L, U, m0, csw):
    """Per-site 12x12 matrix (4 + m0) + c_sw (i/4) sum sigma F (Sec. 1)."""
    L = _dims(L)
    V = int(np.prod(L))
    U = _c128(U)
    A = np.zeros((V, 12, 12), np.complex128)
    _check(lib().oracle_clover(_p(L), _p(U), float(m0), float(csw), _p(A)), "oracle_clover")
    return A


def apply_D(L, U, A, bc, psi, dagger=False):
    """D psi, or D^+ psi written out directly (not via gamma5)."""
    L = _dims(L)
    U, A, psi = _c128(U), _c128(A), _c128(psi)
    out = np.empty_like(psi)
    _check(lib().oracle_apply_D(_p(L), _p(U), _p(A), _p(_bc(bc)), _p(psi), _p(out), int(dagger)),
           "oracle_apply_D")
    return out


def dD_apply(L, U, dU, bc, csw, x):
    """(dD/dh) x for the link deformation U -> U + h dU (first order)."""
    L = _dims(L)
    U, dU, x = _c128(U), _c128(dU), _c128(x)
    out = np.empty_like(x)
    _check(lib().oracle_dD_apply(_p(L), _p(U), _p(dU), _p(_bc(bc)), float(csw), _p(x), _p(out)),
           "oracle_dD_apply")
    return out


def sap(L, U, A, bc, block, eta, ncy, nmr, eo=True, reverse=False, return_rho=False):
    """psi = M_SAP eta (Sec. 4 SAP cycles with MR block solves)."""
    L = _dims(L)
    b = _dims(block)
    U, A, eta = _c128(U), _c128(A), _c128(eta)
    psi = np.empty_like(eta)
    rho = np.empty_like(eta) if return_rho else None
    _check(lib().oracle_sap(_p(L), _p(U), _p(A), _p(_bc(bc)), _p(b), int(ncy), int(nmr), int(eo),
                            int(reverse), _p(eta), _p(psi), _p(rho)), "oracle_sap")
    return (psi, rho) if return_rho else psi


def block_sites(L, block, n):
    L = _dims(L)
    b = _dims(block)
    sites = np.empty(int(np.prod(b)), np.int64)
    _check(lib().oracle_block_sites(_p(L), _p(b), int(n), _p(sites)), "oracle_block_sites")
    return sites


def block_mr(L, U, A, bc, block, n, rho_blk, nmr, eo=True):
    """MR approximation of D_blk^-1 rho for block n (block-ordered arrays)."""
    L = _dims(L)
    b = _dims(block)
    U, A, rho_blk = _c128(U), _c128(A), _c128(rho_blk)
    chi = np.empty_like(rho_blk)
    _check(lib().oracle_block_mr(_p(L), _p(U), _p(A), _p(_bc(bc)), _p(b), int(n), int(nmr), int(eo),
                                 _p(rho_blk), _p(chi)), "oracle_block_mr")
    return chi


def fgcr(L, U, A, bc, b, x0=None, nkv=16, max_restarts=100, tol=1e-12, precond=False,
         block=(2, 2, 2, 2), ncy=4, nmr=4, eo=True, max_iters=0):
    """Solve D x = b by (F)GCR; returns (x, iterations, cycles, converged, true_rel_res).

    max_iters > 0 stops after that many iterations (bounded timing samples)."""
    L = _dims(L)
    bs = _dims(block)
    U, A, b = _c128(U), _c128(A), _c128(b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    info = np.zeros(3, np.int32)
    res = np.zeros(1, np.float64)
    _check(lib().oracle_fgcr(_p(L), _p(U), _p(A), _p(_bc(bc)), _p(b), _p(x), int(nkv),
                             int(max_restarts), float(tol), int(precond), _p(bs), int(ncy), int(nmr),
                             int(eo), int(max_iters), _p(info), _p(res)), "oracle_fgcr")
    return x, int(info[0]), int(info[1]), bool(info[2]), float(res[0])
