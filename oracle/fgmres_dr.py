"""Flexible GMRES with deflated restarts (FGMRES-DR), plain numpy (test
infrastructure only: imported by ``tests/`` and nothing on the product path).

Sec. 4 of the paper: at the end of a flexible GMRES cycle of length m the
harmonic Ritz pairs of the small Arnoldi matrix H are computed; the harmonic
Ritz vectors of the k < m smallest values span the deflation subspace, which,
augmented with the residual, is the starting Krylov subspace of the next cycle
("deflated restarts"; the flexible generalisation of GMRES-DR).

The routine works on flattened complex vectors with caller-supplied operator
``A(v)`` and preconditioner ``M(v)`` (any callables), so it can be pinned on
dense matrices as well as on the lattice operator.  Written from the
definitions, step by step, with numpy's least squares, eigenvalue and QR
routines as the small dense steps:

* Arnoldi with a flexible preconditioner: z_j = M(v_j), w = A z_j, w is
  orthogonalised against v_0..v_j (modified Gram-Schmidt, applied twice),
  h_{j+1,j} = |w|, v_{j+1} = w / |w|; so A Z_m = V_{m+1} Hbar_m.
* Cycle end: y = argmin |c - Hbar_m y| (c = coordinates of the cycle's initial
  residual in V_{m+1}); x += Z_m y; the true residual b - A x decides
  convergence.
* Harmonic Ritz pairs of A on range(Z_m) with respect to range(V): the
  eigenpairs of H_m + |h_{m+1,m}|^2 f e_m^H with f = H_m^{-H} e_m (H_m the
  square top of Hbar_m).  The k eigenvectors g of smallest |theta|, padded
  with a zero row, and the residual coordinates s = c - Hbar_m y form the
  (m+1) x (k+1) matrix P; its QR factor Q gives the new basis V Q, the new
  Z_m Q[:m, :k], the new Hbar = Q^H Hbar_m Q[:m, :k] and the new c = Q^H s.
  The next cycle's Arnoldi steps continue from column k.
"""
from __future__ import annotations

import numpy as np


def fgmres_dr(A, M, b, x0=None, m=16, k=4, tol=1e-12, max_cycles=200, keep_state=False):
    """Solve A x = b.  Returns (x, info) with info = {"cycles", "matvecs",
    "converged", "true_rel_res", "history" (true relative residual per cycle),
    "ritz" (harmonic Ritz values of the last deflated restart)} and, with
    keep_state, "state" = (V, Z, Hbar, c) right after the first deflated
    restart, for checking the Arnoldi-like relation A Z_k = V_{k+1} Hbar_k."""
    if not (0 <= k < m):
        raise ValueError("need 0 <= k < m")
    b = np.asarray(b, np.complex128).ravel()
    n = b.size
    x = np.zeros(n, np.complex128) if x0 is None else np.asarray(x0, np.complex128).ravel().copy()
    bnorm = np.linalg.norm(b)
    r = b - A(x)
    matvecs = 1
    V = np.zeros((n, m + 1), np.complex128)
    Z = np.zeros((n, m), np.complex128)
    H = np.zeros((m + 1, m), np.complex128)
    c = np.zeros(m + 1, np.complex128)
    beta = np.linalg.norm(r)
    info = {"cycles": 0, "matvecs": 0, "converged": beta <= tol * bnorm, "true_rel_res": beta / bnorm,
            "history": [beta / bnorm], "ritz": None}
    if info["converged"]:
        info["matvecs"] = matvecs
        return x, info
    V[:, 0] = r / beta
    c[0] = beta
    j0 = 0
    for cycle in range(max_cycles):
        for j in range(j0, m):
            Z[:, j] = M(V[:, j])
            w = A(Z[:, j])
            matvecs += 1
            for _ in range(2):  # modified Gram-Schmidt, twice
                for i in range(j + 1):
                    h = np.vdot(V[:, i], w)
                    H[i, j] += h
                    w = w - h * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / H[j + 1, j]
        y = np.linalg.lstsq(H, c, rcond=None)[0]
        x = x + Z @ y
        r = b - A(x)
        matvecs += 1
        res = np.linalg.norm(r) / bnorm
        info["cycles"] = cycle + 1
        info["history"].append(res)
        info["true_rel_res"] = res
        if res <= tol:
            info["converged"] = True
            break
        s = c - H @ y
        if k == 0:  # plain restart from the true residual
            beta = np.linalg.norm(r)
            V[:] = 0
            Z[:] = 0
            H[:] = 0
            c[:] = 0
            V[:, 0] = r / beta
            c[0] = beta
            j0 = 0
            continue
        Hm = H[:m, :m]
        em = np.zeros(m, np.complex128)
        em[-1] = 1.0
        f = np.linalg.solve(Hm.conj().T, em)
        G = Hm + abs(H[m, m - 1]) ** 2 * np.outer(f, em)
        theta, g = np.linalg.eig(G)
        order = np.argsort(np.abs(theta))[:k]
        info["ritz"] = theta[order]
        P = np.zeros((m + 1, k + 1), np.complex128)
        P[:m, :k] = g[:, order]
        P[:, k] = s
        Q, _ = np.linalg.qr(P)
        Vn = V @ Q
        Zn = Z @ Q[:m, :k]
        Hn = Q.conj().T @ H @ Q[:m, :k]
        c = Q.conj().T @ s
        V[:] = 0
        Z[:] = 0
        H[:] = 0
        V[:, :k + 1] = Vn
        Z[:, :k] = Zn
        H[:k + 1, :k] = Hn
        c = np.concatenate([c, np.zeros(m - k, np.complex128)])
        j0 = k
        if keep_state and "state" not in info:
            info["state"] = (V[:, :k + 1].copy(), Z[:, :k].copy(), H[:k + 1, :k].copy(), c[:k + 1].copy())
    info["matvecs"] = matvecs
    return x, info
