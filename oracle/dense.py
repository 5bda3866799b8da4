"""Independent dense numpy assembly of the clover Wilson-Dirac matrix.

Test infrastructure only.  This module re-derives the operator of Sec. 1/4
(Wilson-Dirac with clover term) from scratch -- gamma matrices built from the
Pauli matrices, plaquettes from rolled numpy fields, hopping terms as dense
matrix blocks -- so that it shares no code with ``oracle.c`` and can pin it on
tiny lattices (2^4: a 192 x 192 matrix; 4^4: 3072 x 3072).
"""
from __future__ import annotations

import numpy as np

PAULI = [np.array([[0, 1], [1, 0]], complex),
         np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex)]


def gammas():
    """Chiral (Weyl) basis: g0 = [[0, -1], [-1, 0]], g_k = [[0, -i s_k], [i s_k, 0]]."""
    z = np.zeros((2, 2), complex)
    one = np.eye(2)
    g = [np.block([[z, -one], [-one, z]])]
    for s in PAULI:
        g.append(np.block([[z, -1j * s], [1j * s, z]]))
    return g


def _lattice_links(L, U):
    """U reshaped to (L0, L1, L2, L3, 4, 3, 3)."""
    return np.asarray(U, complex).reshape(tuple(L) + (4, 3, 3))


def _fwd(field, mu):
    """field(x + mu) as a field over x (periodic)."""
    return np.roll(field, -1, axis=mu)


def _bwd(field, mu):
    return np.roll(field, 1, axis=mu)


def _mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.einsum("...ab,...bc->...ac", out, m)
    return out


def _dg(m):
    return np.conj(np.swapaxes(m, -1, -2))


def field_strength(L, U):
    """Fhat[mu][nu] as (L0..L3, 3, 3) arrays, from the four counter-clockwise leaves."""
    W = _lattice_links(L, U)
    F = [[None] * 4 for _ in range(4)]
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                F[mu][nu] = np.zeros(tuple(L) + (3, 3), complex)
                continue
            Umu, Unu = W[..., mu, :, :], W[..., nu, :, :]
            # plaquette P(y) = U_mu(y) U_nu(y+mu) U_mu(y+nu)^+ U_nu(y)^+
            P = _mm(Umu, _fwd(Unu, mu), _dg(_fwd(Umu, nu)), _dg(Unu))
            # the leaves at x are P(x), P(x-mu), P(x-nu), P(x-mu-nu) rotated to start at x
            Pm = _bwd(P, mu)
            Umu_m = _bwd(Umu, mu)                       # U_mu(x - mu)
            leaf2 = _mm(_dg(Umu_m), Pm, Umu_m)
            Pn = _bwd(P, nu)
            Unu_n = _bwd(Unu, nu)                       # U_nu(x - nu)
            leaf4 = _mm(_dg(Unu_n), Pn, Unu_n)
            Pmn = _bwd(Pm, nu)
            T = _mm(_dg(Umu_m), _dg(_bwd(Unu_n, mu)))   # U_mu(x-mu)^+ U_nu(x-mu-nu)^+
            leaf3 = _mm(T, Pmn, _dg(T))
            Q = P + leaf2 + leaf3 + leaf4
            F[mu][nu] = (Q - _dg(Q)) / 8.0
    return F


def clover_blocks(L, U, m0, csw):
    """Per-site 12x12 clover matrices (V, 12, 12), index spin*3 + colour."""
    g = gammas()
    F = field_strength(L, U)
    V = int(np.prod(L))
    A = np.zeros((V, 12, 12), complex)
    A[:] = (4.0 + m0) * np.eye(12)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            sig = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
            Fm = F[mu][nu].reshape(V, 3, 3)
            A += csw * 0.25j * np.einsum("st,vab->vsatb", sig, Fm).reshape(V, 12, 12)
    return A


def dirac_matrix(L, U, m0, csw, bc):
    """Dense 12V x 12V matrix of D (row = site*12 + spin*3 + colour)."""
    L = list(L)
    V = int(np.prod(L))
    g = gammas()
    W = np.asarray(U, complex).reshape(V, 4, 3, 3)
    A = clover_blocks(L, U, m0, csw)
    D = np.zeros((12 * V, 12 * V), complex)
    coords = np.array(np.unravel_index(np.arange(V), L)).T
    strides = [L[1] * L[2] * L[3], L[2] * L[3], L[3], 1]
    one4 = np.eye(4)
    for x in range(V):
        D[12 * x:12 * x + 12, 12 * x:12 * x + 12] += A[x]
        c = coords[x]
        for mu in range(4):
            up = c.copy()
            up[mu] = (c[mu] + 1) % L[mu]
            dn = c.copy()
            dn[mu] = (c[mu] - 1) % L[mu]
            y = int(np.dot(up, strides))
            z = int(np.dot(dn, strides))
            s_up = bc[mu] if c[mu] == L[mu] - 1 else 1.0     # hop x -> x+mu wraps
            s_dn = bc[mu] if c[mu] == 0 else 1.0              # hop x-mu -> x wraps
            D[12 * x:12 * x + 12, 12 * y:12 * y + 12] += -0.5 * s_up * np.kron(one4 - g[mu], W[x, mu])
            D[12 * x:12 * x + 12, 12 * z:12 * z + 12] += -0.5 * s_dn * np.kron(one4 + g[mu], _dg(W[z, mu]))
    return D
