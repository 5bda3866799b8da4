"""Pins for the oracle's CG on the normal equations (the CG fallback that
Sec. 4 foresees for the hardest cases).

* the residuals of CG on D^+ D are mutually orthogonal (A-conjugate search
  directions give orthogonal residuals);
* on a Hermitian positive definite matrix with n distinct eigenvalues CG
  terminates in at most n steps (exact arithmetic; here to rounding);
* on the lattice operator the solution equals dense LU of the
  independently assembled D.
"""
import numpy as np

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


def test_residuals_are_orthogonal(orc):
    from oracle.cgne import cgne
    dims, U, A, b, w = _lat44()
    D = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape)).ravel()
    Dh = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape), dagger=True).ravel()
    x, info = cgne(D, Dh, b, tol=1e-30, max_iter=8)
    R = np.stack(info["residuals"], axis=1)
    G = R.conj().T @ R
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) <= 1e-10 * np.max(np.abs(np.diag(G)))


def test_finite_termination_on_small_spectrum():
    """A = S diag(sigma) S^-1 with 6 distinct singular values: D^+ D has 6
    distinct eigenvalues, so CGNE reaches the solution in 6 steps."""
    from oracle.cgne import cgne
    rng = np.random.default_rng(4)
    n = 60
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    sig = np.repeat([0.5, 1.0, 1.5, 2.0, 3.0, 4.0], 10)
    M = Q1 @ np.diag(sig) @ Q2.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = cgne(lambda v: M @ v, lambda v: M.conj().T @ v, b, tol=1e-11, max_iter=40)
    assert info["converged"] and info["iterations"] <= 7
    assert rel(x, np.linalg.solve(M, b)) < 1e-10


def test_solution_matches_dense_lu(orc):
    from oracle import dense
    from oracle.cgne import cgne
    dims, U, A, b, w = _lat44()
    Dm = dense.dirac_matrix(dims, U, w["m0"], w["csw"], AP)
    D = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape)).ravel()
    Dh = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape), dagger=True).ravel()
    x, info = cgne(D, Dh, b, tol=1e-12, max_iter=2000)
    assert info["converged"]
    assert rel(x, np.linalg.solve(Dm, b.ravel())) < 1e-10
