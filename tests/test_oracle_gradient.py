"""Pins for the oracle's operator derivative and fermion force (CPU).

The inversions feed the HMC fermion force (Sec. 1).  For the link deformation
U_mu(x) -> exp(i h theta_a lambda_a / 2) U_mu(x) the oracle's dD/dh is
checked against central finite differences of D itself, and the force
dL/dh = -Re(y^+ dD x) (L = Re(phi^+ D^-1 phi), y = D^-+ phi) against central
finite differences of L computed from full re-solves.
"""
import numpy as np
import pytest

from helpers import g5, rel, vdot
from paper_1109_4279_gb300 import synth

AP = synth.ANTIPERIODIC_T


def _deform(U, theta_field, h):
    """U -> exp(i h sum_a theta_a lambda_a / 2) U for every link (theta (V,4,8))."""
    return np.einsum("vmab,vmbc->vmac", synth.su3_exp(h * synth.algebra(theta_field)), U)


def _dU(U, theta_field):
    return np.einsum("vmab,vmbc->vmac", 1j * synth.algebra(theta_field), U)


@pytest.mark.parametrize("single", [True, False])
def test_dD_matches_finite_difference(orc, single):
    dims = (4, 2, 4, 2)
    m0, csw = 0.05, 1.5
    U, rng = synth.gauge_field(dims, 0.5, 31)
    V = synth.volume(dims)
    x = synth.gaussian_spinor(dims, rng)
    th = np.zeros((V, 4, 8))
    if single:
        th[5, 2] = rng.standard_normal(8)
    else:
        th = rng.standard_normal((V, 4, 8))
    h = 1e-5
    Dx = []
    for s in (+1, -1):
        Uh = _deform(U, th, s * h)
        Dx.append(orc.apply_D(dims, Uh, orc.clover(dims, Uh, m0, csw), AP, x))
    fd = (Dx[0] - Dx[1]) / (2 * h)
    an = orc.dD_apply(dims, U, _dU(U, th), AP, csw, x)
    assert rel(an, fd) < 1e-8
    # the clover part is really exercised: csw = 0 gives a different answer
    an0 = orc.dD_apply(dims, U, _dU(U, th), AP, 0.0, x)
    assert rel(an0, an) > 1e-3


def test_force_matches_finite_difference_of_solves(orc):
    """dL/dh for 4 random single-link directions and one global direction."""
    dims = (2, 2, 2, 4)
    m0, csw = 0.1, 1.2
    U, rng = synth.gauge_field(dims, 0.5, 41)
    V = synth.volume(dims)
    phi = synth.gaussian_spinor(dims, rng)

    def solve(Uh, rhs):
        A = orc.clover(dims, Uh, m0, csw)
        x, _, _, conv, res = orc.fgcr(dims, Uh, A, AP, rhs, nkv=32, tol=1e-14, max_restarts=200)
        assert conv
        return x

    x = solve(U, phi)
    y = g5(solve(U, g5(phi)))   # D^-+ = g5 D^-1 g5
    A = orc.clover(dims, U, m0, csw)
    assert rel(orc.apply_D(dims, U, A, AP, y, dagger=True), phi) < 1e-12
    sites, mus, thetas = synth.link_directions(dims, 4, seed=1005)
    dirs = []
    for s, m, t in zip(sites, mus, thetas):
        th = np.zeros((V, 4, 8))
        th[s, m] = t
        dirs.append(th)
    dirs.append(rng.standard_normal((V, 4, 8)))
    h = 1e-4
    for th in dirs:
        an = -np.real(vdot(y, orc.dD_apply(dims, U, _dU(U, th), AP, csw, x)))
        L = [np.real(vdot(phi, solve(_deform(U, th, s * h), phi))) for s in (+1, -1)]
        fd = (L[0] - L[1]) / (2 * h)
        assert abs(an - fd) <= 1e-7 * max(1.0, abs(fd)), (an, fd)


def test_dL_dphi_is_x_plus_y(orc):
    """For L = Re(phi^+ D^-1 phi) the gradient d/dRe + i d/dIm equals x + y."""
    dims = (2, 2, 2, 2)
    U, rng = synth.gauge_field(dims, 0.5, 51)
    phi = synth.gaussian_spinor(dims, rng)
    A = orc.clover(dims, U, 0.2, 1.0)

    def L(p):
        x, *_ = orc.fgcr(dims, U, A, AP, p, nkv=32, tol=1e-14, max_restarts=200)
        return np.real(vdot(p, x))

    x, *_ = orc.fgcr(dims, U, A, AP, phi, nkv=32, tol=1e-14, max_restarts=200)
    y = g5(orc.fgcr(dims, U, A, AP, g5(phi), nkv=32, tol=1e-14, max_restarts=200)[0])
    g = x + y
    for _ in range(3):
        d = synth.gaussian_spinor(dims, rng)
        h = 1e-5
        fd = (L(phi + h * d) - L(phi - h * d)) / (2 * h)
        assert abs(fd - np.real(vdot(d, g))) < 1e-7 * abs(fd)
