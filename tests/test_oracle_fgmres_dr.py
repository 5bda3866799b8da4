"""Pins for the oracle's FGMRES-DR (Sec. 4: flexible GMRES with deflated
restarts from the harmonic Ritz vectors of the smallest k values).

* k = 0 without preconditioner is restarted GMRES, whose iterates equal those
  of GCR over the same Krylov space: one cycle of length m against m GCR
  iterations of the C oracle;
* after a deflated restart the kept basis satisfies A Z_k = V_{k+1} Hbar_k;
* on a matrix with a known spectrum (a few tiny isolated eigenvalues), the
  harmonic Ritz values converge to exactly those eigenvalues, and deflation
  beats plain restarts, which stall;
* with the (non-linear) SAP preconditioner the solve reaches the dense LU
  solution of the independently assembled operator.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

AP = synth.ANTIPERIODIC_T


def _lat44():
    import oracle
    w = synth.WORKLOADS["4^4 fp64"]
    dims = w["dims"]
    U, rng = synth.gauge_field(dims, w["eps"], w["seed"])
    b = synth.gaussian_spinor(dims, rng)
    A = oracle.clover(dims, U, w["m0"], w["csw"])
    return dims, U, A, b, w


def test_k0_unpreconditioned_equals_gcr(orc):
    """One GMRES(12) cycle = 12 GCR steps (the same minimal-residual iterate)."""
    from oracle.fgmres_dr import fgmres_dr
    dims, U, A, b, w = _lat44()
    op = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape)).ravel()
    x, info = fgmres_dr(op, lambda v: v, b, m=12, k=0, tol=1e-30, max_cycles=1)
    x_gcr, it, *_ = orc.fgcr(dims, U, A, AP, b, nkv=12, max_restarts=1, tol=1e-30, precond=False, max_iters=12)
    assert it == 12 and info["cycles"] == 1
    assert rel(x, x_gcr.ravel()) < 1e-10


def test_arnoldi_relation_after_deflated_restart(orc):
    from oracle.fgmres_dr import fgmres_dr
    dims, U, A, b, w = _lat44()
    op = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape)).ravel()
    sap = lambda v: orc.sap(dims, U, A, AP, w["block"], v.reshape(b.shape), 2, 2).ravel()
    x, info = fgmres_dr(op, sap, b, m=8, k=3, tol=1e-30, max_cycles=2, keep_state=True)
    V, Z, Hk, c = info["state"]
    AZ = np.stack([op(Z[:, j]) for j in range(Z.shape[1])], axis=1)
    # exact in exact arithmetic: the harmonic Ritz residuals and the least-squares
    # residual all lie in the one-dimensional complement of range(Hbar_m); the
    # bound allows for the conditioning of the small non-normal eigenproblem
    assert np.linalg.norm(AZ - V @ Hk) <= 1e-10 * np.linalg.norm(Hk)
    assert np.linalg.norm(V.conj().T @ V - np.eye(V.shape[1])) < 1e-12
    # c holds the coordinates of the current residual: |c| = |b - A x_1|
    assert abs(np.linalg.norm(c) - info["history"][1] * np.linalg.norm(b)) <= 1e-10 * np.linalg.norm(b)


def _known_spectrum(n=240, tiny=(1e-3, 2e-3 + 1e-3j, 4e-3 - 2e-3j), seed=3):
    rng = np.random.default_rng(seed)
    lam = np.concatenate([np.array(tiny, np.complex128),
                          1.0 + rng.random(n - len(tiny)) + 0.3j * (rng.random(n - len(tiny)) - 0.5)])
    S = np.eye(n) + 0.1 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    A = S @ np.diag(lam) @ np.linalg.inv(S)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b, np.array(tiny, np.complex128)


def test_harmonic_ritz_values_find_the_small_eigenvalues():
    from oracle.fgmres_dr import fgmres_dr
    A, b, tiny = _known_spectrum()
    x, info = fgmres_dr(lambda v: A @ v, lambda v: v, b, m=20, k=5, tol=1e-12, max_cycles=200)
    assert info["converged"]
    assert rel(x, np.linalg.solve(A, b)) < 1e-8
    # deflation against plain restarts with the same number of vectors
    _, plain = fgmres_dr(lambda v: A @ v, lambda v: v, b, m=20, k=0, tol=1e-12, max_cycles=200)
    assert info["matvecs"] * 2 < plain["matvecs"]
    # three deflated cycles past convergence: each tiny eigenvalue is matched
    # by a harmonic Ritz value to rounding level
    _, info = fgmres_dr(lambda v: A @ v, lambda v: v, b, m=20, k=5, tol=0.0, max_cycles=3)
    for t in tiny:
        assert np.min(np.abs(info["ritz"] - t)) < 1e-9 * abs(t)


def test_sap_preconditioned_solution_matches_dense_lu(orc):
    from oracle import dense
    from oracle.fgmres_dr import fgmres_dr
    dims, U, A, b, w = _lat44()
    D = dense.dirac_matrix(dims, U, w["m0"], w["csw"], AP)
    op = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape)).ravel()
    sap = lambda v: orc.sap(dims, U, A, AP, w["block"], v.reshape(b.shape), 4, 4).ravel()
    x, info = fgmres_dr(op, sap, b, m=8, k=3, tol=1e-12, max_cycles=50)
    assert info["converged"] and info["true_rel_res"] <= 1e-12
    assert rel(x, np.linalg.solve(D, b.ravel())) < 1e-10


def test_rejects_bad_sizes():
    from oracle.fgmres_dr import fgmres_dr
    with pytest.raises(ValueError):
        fgmres_dr(lambda v: v, lambda v: v, np.ones(4), m=4, k=4)
