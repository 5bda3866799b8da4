"""Even/odd preconditioning of the Wilson-Dirac operator over the whole
lattice (the Schur complement on the even sites), plain numpy over the C
oracle's operator (test infrastructure only).

Sec. 4 foresees CG for the most difficult cases; the classic companion of CG
is the even/odd split of the global operator.  Sites split by the parity of
x0 + x1 + x2 + x3.  Writing D = [[A_ee, D_eo], [D_oe, A_oo]] (A the per-site
term 4 + m0 + clover, D_eo and D_oe the hops between the parities),
D x = b is equivalent to

  Dhat x_e = bhat_e,   Dhat = A_ee - D_eo A_oo^-1 D_oe,
  bhat_e = b_e - D_eo A_oo^-1 b_o,
  x_o = A_oo^-1 (b_o - D_oe x_e),

and the residual of the whole system is b - D x = (bhat_e - Dhat x_e, 0).
Each piece here is a full-lattice application of the oracle's D to a field
that vanishes on one parity: for y zero on the odd sites, (D y)_e = A_ee y_e
and (D y)_o = D_oe y_e (likewise with the parities exchanged).  The adjoint
Dhat^+ has the same form with D^+ in place of D (A is Hermitian).
"""
from __future__ import annotations

import numpy as np

from . import cgne


def parity(L):
    """0 on even sites, 1 on odd sites, lexicographic (x0 slowest)."""
    c = np.indices(tuple(L)).sum(axis=0) % 2
    return c.ravel()


def odd_inverse(A, L):
    """A_oo^-1 as an array of the odd sites' inverted 12x12 matrices (zero
    matrices on even sites), from the oracle's per-site clover A."""
    odd = parity(L) == 1
    inv = np.zeros_like(A)
    inv[odd] = np.linalg.inv(A[odd])
    return inv


def _apply_site(M, psi):
    V = M.shape[0]
    return np.einsum("vij,vj->vi", M, psi.reshape(V, 12)).reshape(psi.shape)


def _mask(psi, L, p):
    return psi * (parity(L) == p)[:, None, None]


def schur(orc, L, U, A, bc, Ainv, x, dagger=False):
    """Dhat x_e (or Dhat^+ x_e); x is a full field of which only the even sites
    are read; the result vanishes on the odd sites."""
    y = _mask(np.asarray(x, np.complex128), L, 0)
    Dy = orc.apply_D(L, U, A, bc, y, dagger=dagger)      # (A_ee y_e, D_oe y_e)
    z = _apply_site(Ainv, _mask(Dy, L, 1))                # (0, A_oo^-1 D_oe y_e)
    Dz = orc.apply_D(L, U, A, bc, z, dagger=dagger)      # even part: D_eo A_oo^-1 D_oe y_e
    return _mask(Dy - Dz, L, 0)


def rhs(orc, L, U, A, bc, Ainv, b):
    """bhat_e = b_e - D_eo A_oo^-1 b_o (zero on the odd sites)."""
    z = _apply_site(Ainv, _mask(np.asarray(b, np.complex128), L, 1))
    return _mask(b - orc.apply_D(L, U, A, bc, z), L, 0)


def reconstruct(orc, L, U, A, bc, Ainv, b, x):
    """The full solution from its even part: x_o = A_oo^-1 (b_o - D_oe x_e)."""
    xe = _mask(np.asarray(x, np.complex128), L, 0)
    t = _mask(b - orc.apply_D(L, U, A, bc, xe), L, 1)
    return xe + _apply_site(Ainv, t)


def cg_eo(orc, L, U, A, bc, b, tol=1e-12, max_iter=20000):
    """Solve D x = b by CG on Dhat^+ Dhat x_e = Dhat^+ bhat_e (the textbook
    steps of `cgne.cgne`), stopping when |bhat_e - Dhat x_e| <= tol |b|, the
    whole system's residual; then reconstruct the odd sites.  Returns
    (x, info) with cgne's info."""
    b = np.asarray(b, np.complex128)
    Ainv = odd_inverse(A, L)
    bh = rhs(orc, L, U, A, bc, Ainv, b)
    shape = b.shape

    def Dh(v):
        return schur(orc, L, U, A, bc, Ainv, v.reshape(shape)).ravel()

    def Dhd(v):
        return schur(orc, L, U, A, bc, Ainv, v.reshape(shape), dagger=True).ravel()

    scale = np.linalg.norm(b) / np.linalg.norm(bh)
    xe, info = cgne.cgne(Dh, Dhd, bh.ravel(), tol=tol * scale, max_iter=max_iter)
    return reconstruct(orc, L, U, A, bc, Ainv, b, xe.reshape(shape)), info
