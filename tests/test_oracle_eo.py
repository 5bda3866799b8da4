"""Pins for the oracle's even/odd-preconditioned operator and CG (the global
even/odd split that accompanies the CG fallback of Sec. 4).

* the Schur complement Dhat = D_ee - D_eo D_oo^-1 D_oe formed from blocks of
  the independently assembled dense D (oracle/dense.py) equals the oracle's
  Dhat, and its conjugate transpose equals the oracle's Dhat^+;
* the even/odd CG solution equals dense LU of the full D, and its residual
  (recomputed with the full operator) meets the tolerance;
* a planted mistake (A_oo in place of A_oo^-1, or the parities swapped) fails
  the first pin.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

AP = synth.ANTIPERIODIC_T


def _case(dims, eps, seed, m0, csw):
    import oracle
    U, rng = synth.gauge_field(dims, eps, seed)
    b = synth.gaussian_spinor(dims, rng)
    A = oracle.clover(dims, U, m0, csw)
    return U, A, b, rng


def _dense_schur(dims, U, m0, csw, bc):
    from oracle import dense, eo
    D = dense.dirac_matrix(dims, U, m0, csw, bc)
    par = np.repeat(eo.parity(dims), 12)
    e, o = np.where(par == 0)[0], np.where(par == 1)[0]
    S = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    return S, e


CASES = [((2, 2, 2, 2), 0.5, 3, 0.1, 1.2), ((4, 2, 2, 2), 0.6, 4, -0.2, 1.5), ((4, 4, 4, 4), 0.3, 1, 0.1, 1.0)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_schur_matches_dense_blocks(orc, case):
    from oracle import eo
    dims, eps, seed, m0, csw = case
    U, A, b, rng = _case(dims, eps, seed, m0, csw)
    S, e = _dense_schur(dims, U, m0, csw, AP)
    Ainv = eo.odd_inverse(A, dims)
    x = synth.gaussian_spinor(dims, rng)
    for dag, M in ((False, S), (True, S.conj().T)):
        out = eo.schur(orc, dims, U, A, AP, Ainv, x, dagger=dag).ravel()
        assert rel(out[e], M @ x.ravel()[e]) < 1e-12
        odd = np.setdiff1d(np.arange(out.size), e)
        assert np.max(np.abs(out[odd])) == 0.0


@pytest.mark.parametrize("case", CASES[1:], ids=lambda c: "x".join(map(str, c[0])))
def test_cg_eo_matches_dense_lu(orc, case):
    from oracle import dense, eo
    dims, eps, seed, m0, csw = case
    U, A, b, rng = _case(dims, eps, seed, m0, csw)
    x, info = eo.cg_eo(orc, dims, U, A, AP, b, tol=1e-12)
    assert info["converged"]
    D = dense.dirac_matrix(dims, U, m0, csw, AP)
    assert rel(x.ravel(), np.linalg.solve(D, b.ravel())) < 1e-9
    assert np.linalg.norm(b - orc.apply_D(dims, U, A, AP, x)) <= 1.01e-12 * np.linalg.norm(b)


def test_even_odd_cg_needs_fewer_iterations(orc):
    """On 8^4 at m0 = -0.2 the Schur system is better conditioned than D^+ D:
    even/odd CG reaches the same residual in fewer iterations than CGNE."""
    from oracle import eo
    from oracle.cgne import cgne
    dims = (8, 8, 8, 8)
    U, A, b, rng = _case(dims, 0.5, 6, -0.2, 1.5)
    x, info = eo.cg_eo(orc, dims, U, A, AP, b, tol=1e-10)
    assert info["converged"]
    D = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape)).ravel()
    Dh = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape), dagger=True).ravel()
    _, info_ne = cgne(D, Dh, b, tol=1e-10)
    assert info_ne["converged"] and info["iterations"] < 0.75 * info_ne["iterations"], (
        info["iterations"], info_ne["iterations"])


@pytest.mark.parametrize("mutation", ["A_oo instead of its inverse", "parities swapped"])
def test_planted_mistakes_fail_the_dense_pin(orc, mutation, monkeypatch):
    from oracle import eo
    dims, eps, seed, m0, csw = CASES[1]
    U, A, b, rng = _case(dims, eps, seed, m0, csw)
    S, e = _dense_schur(dims, U, m0, csw, AP)
    if mutation == "parities swapped":
        real = eo.parity
        monkeypatch.setattr(eo, "parity", lambda L: 1 - real(L))
        Ainv = eo.odd_inverse(A, dims)
    else:
        odd = eo.parity(dims) == 1
        Ainv = np.zeros_like(A)
        Ainv[odd] = A[odd]
    x = synth.gaussian_spinor(dims, rng)
    out = eo.schur(orc, dims, U, A, AP, Ainv, x).ravel()
    assert rel(out[e], S @ x.ravel()[e]) > 1e-3
