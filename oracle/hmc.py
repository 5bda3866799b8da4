"""Hybrid Monte Carlo molecular-dynamics trajectory for two degenerate
clover-Wilson flavours, plain numpy (test infrastructure only).

The paper's inversions exist to feed the HMC fermion force (Sec. 1).  The
trajectory written out here, step by step:

* fields: links U (V,4,3,3) lexicographic, momenta pi (V,4,8) with
  P = sum_a pi_a lambda_a / 2; pseudofermion phi = D^+ eta from a Gaussian eta;
* H = 1/2 sum pi_a^2 + S_g + S_f, with the Wilson plaquette action
  S_g = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3) and S_f = phi^+ (D^+ D)^-1 phi
  = |Y|^2, Y = D^-+ phi;
* forces F_a(x, mu) = dS/dtheta_a for U_mu(x) -> exp(i theta_a lambda_a/2) U_mu(x):
  gauge part (beta/6) Im tr(lambda_a U_mu(x) V_mu(x)) with V the sum of the six
  staples; fermion part -2 Re(Y^+ (dD/dtheta_a) X) with X = D^-1 Y;
* leapfrog: pi -= eps/2 F; n times { U <- exp(i eps P) U; pi -= eps F }, the last
  momentum step a half step; Metropolis with exp(-dH).

Library primitives used as steps: scipy's matrix exponential, the C oracle's
operator, clover, dD/dtheta and GCR solve.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

# Gell-Mann matrices, written out
_L = np.zeros((8, 3, 3), np.complex128)
_L[0][0, 1] = _L[0][1, 0] = 1
_L[1][0, 1], _L[1][1, 0] = -1j, 1j
_L[2][0, 0], _L[2][1, 1] = 1, -1
_L[3][0, 2] = _L[3][2, 0] = 1
_L[4][0, 2], _L[4][2, 0] = -1j, 1j
_L[5][1, 2] = _L[5][2, 1] = 1
_L[6][1, 2], _L[6][2, 1] = -1j, 1j
_L[7][0, 0] = _L[7][1, 1] = 1 / np.sqrt(3)
_L[7][2, 2] = -2 / np.sqrt(3)
LAMBDA = _L


def _field(U, dims):
    return U.reshape(tuple(dims) + (4, 3, 3))


def _shift(F, mu, s):
    """F(x + s mu) for a field indexed [x0, x1, x2, x3, ...] (periodic)."""
    return np.roll(F, -s, axis=mu)


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def plaquette_action(U, dims, beta):
    Uf = _field(U, dims)
    S = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um, Un = Uf[..., mu, :, :], Uf[..., nu, :, :]
            P = Um @ _shift(Un, mu, 1) @ _dag(_shift(Um, nu, 1)) @ _dag(Un)
            S += np.sum(1.0 - np.trace(P, axis1=-2, axis2=-1).real / 3.0)
    return beta * S


def staples(U, dims):
    """V_mu(x) = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)."""
    Uf = _field(U, dims)
    out = np.zeros_like(Uf)
    for mu in range(4):
        Um = Uf[..., mu, :, :]
        for nu in range(4):
            if nu == mu:
                continue
            Un = Uf[..., nu, :, :]
            up = _shift(Un, mu, 1) @ _dag(_shift(Um, nu, 1)) @ _dag(Un)
            Un_m = _shift(Un, nu, -1)
            dn = _dag(_shift(Un_m, mu, 1)) @ _dag(_shift(Um, nu, -1)) @ Un_m
            out[..., mu, :, :] += up + dn
    return out.reshape(U.shape)


def gauge_force(U, dims, beta):
    M = np.einsum("vmab,vmbc->vmac", U, staples(U, dims))
    return (beta / 6.0) * np.einsum("aij,vmji->vma", LAMBDA, M).imag


def link_update(U, pi, eps):
    P = np.einsum("vma,aij->vmij", pi, LAMBDA) / 2.0
    E = np.array([expm(1j * eps * p) for p in P.reshape(-1, 3, 3)]).reshape(P.shape)
    return np.einsum("vmab,vmbc->vmac", E, U)


def fermion_force(orc, dims, U, A, bc, csw, X, Y):
    """-2 Re(Y^+ dD/dtheta_a X) for every link and generator (one dD apply each)."""
    V = U.shape[0]
    F = np.zeros((V, 4, 8))
    dU = np.zeros_like(U)
    for x in range(V):
        for mu in range(4):
            for a in range(8):
                dU[x, mu] = 1j * (LAMBDA[a] / 2.0) @ U[x, mu]
                dDX = orc.dD_apply(dims, U, dU, bc, csw, X)
                F[x, mu, a] = -2.0 * np.vdot(Y, dDX).real
            dU[x, mu] = 0
    return F


def _solve(orc, dims, U, A, bc, b, dagger, tol):
    if dagger:  # D^+ = g5 D g5 in the chiral basis
        g5 = np.array([1, 1, -1, -1])[None, :, None]
        x, _, _, conv, _ = orc.fgcr(dims, U, A, bc, g5 * b, nkv=32, max_restarts=500, tol=tol)
        return g5 * x
    x, _, _, conv, _ = orc.fgcr(dims, U, A, bc, b, nkv=32, max_restarts=500, tol=tol)
    return x


def hamiltonian_parts(orc, dims, U, pi, phi, beta, m0, csw, bc, tol):
    A = orc.clover(dims, U, m0, csw)
    Y = _solve(orc, dims, U, A, bc, phi, True, tol)
    return 0.5 * np.sum(pi ** 2), plaquette_action(U, dims, beta), np.vdot(Y, Y).real


def force(orc, dims, U, phi, beta, m0, csw, bc, tol):
    A = orc.clover(dims, U, m0, csw)
    Y = _solve(orc, dims, U, A, bc, phi, True, tol)
    X = _solve(orc, dims, U, A, bc, Y, False, tol)
    return gauge_force(U, dims, beta) + fermion_force(orc, dims, U, A, bc, csw, X, Y)


def trajectory(orc, dims, U, pi, eta, beta, m0, csw, bc, eps, nsteps, tol=1e-13):
    """Returns (U_new, pi_new, H0, H1, (kin, S_g, S_f) at both ends)."""
    A0 = orc.clover(dims, U, m0, csw)
    phi = orc.apply_D(dims, U, A0, bc, eta, dagger=True)
    h0 = hamiltonian_parts(orc, dims, U, pi, phi, beta, m0, csw, bc, tol)
    pi = pi - 0.5 * eps * force(orc, dims, U, phi, beta, m0, csw, bc, tol)
    for s in range(nsteps):
        U = link_update(U, pi, eps)
        step = eps if s < nsteps - 1 else 0.5 * eps
        pi = pi - step * force(orc, dims, U, phi, beta, m0, csw, bc, tol)
    h1 = hamiltonian_parts(orc, dims, U, pi, phi, beta, m0, csw, bc, tol)
    return U, pi, sum(h0), sum(h1), (h0, h1)
