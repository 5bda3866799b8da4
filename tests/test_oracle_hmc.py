"""Pins for the oracle's HMC trajectory (the force the paper's inversions
feed, Sec. 1): plaquette action closed form and gauge invariance, gauge and
fermion forces against finite differences of the actions, reversibility of
the leapfrog trajectory, and the second-order scaling of dH with the step.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

AP = synth.ANTIPERIODIC_T
DIMS = (4, 4, 4, 4)
V = 256


def _deform(U, th, h):
    return np.einsum("vmab,vmbc->vmac", synth.su3_exp(h * synth.algebra(th)), U)


def test_plaquette_action_abelian_closed_form():
    """U_1(x) = exp(i c x_2 lambda_3 / 2), c = 4 pi / L_2 (periodic in x_2), all other links 1:
    every (1,2) plaquette is diag(e^{-ic/2}, e^{ic/2}, 1), the others are 1, so
    S_g = beta V (1 - (1 + 2 cos(c/2)) / 3)."""
    from oracle import hmc
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[:] = np.eye(3)
    c = 4 * np.pi / DIMS[2]
    x2 = np.indices(DIMS).reshape(4, -1)[2]
    U[:, 1, 0, 0] = np.exp(0.5j * c * x2)
    U[:, 1, 1, 1] = np.exp(-0.5j * c * x2)
    beta = 5.3
    S = hmc.plaquette_action(U, DIMS, beta)
    assert abs(S - beta * V * (1 - (1 + 2 * np.cos(c / 2)) / 3)) < 1e-10 * beta * V
    assert abs(hmc.plaquette_action(synth.unit_gauge(DIMS), DIMS, beta)) < 1e-12


def test_plaquette_action_gauge_invariant():
    from oracle import hmc
    U, rng = synth.gauge_field(DIMS, 0.5, 3)
    G = synth.random_su3(V, rng)
    Gf = G.reshape(DIMS + (3, 3))
    Ut = U.copy()
    for mu in range(4):
        Gs = np.roll(Gf, -1, axis=mu).reshape(V, 3, 3)
        Ut[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(Gs, -1, -2))
    assert abs(hmc.plaquette_action(Ut, DIMS, 5.0) - hmc.plaquette_action(U, DIMS, 5.0)) < 1e-10


def test_gauge_force_matches_finite_difference():
    from oracle import hmc
    U, rng = synth.gauge_field(DIMS, 0.5, 5)
    F = hmc.gauge_force(U, DIMS, 5.0)
    for single in (True, False):
        th = np.zeros((V, 4, 8))
        if single:
            th[37, 1] = rng.standard_normal(8)
        else:
            th = rng.standard_normal((V, 4, 8))
        h = 1e-5
        fd = (hmc.plaquette_action(_deform(U, th, h), DIMS, 5.0)
              - hmc.plaquette_action(_deform(U, th, -h), DIMS, 5.0)) / (2 * h)
        assert abs(fd - np.sum(F * th)) < 1e-7 * max(1.0, abs(fd))


def test_fermion_force_matches_finite_difference(orc):
    """dS_f/dh along one link direction, S_f = |D^-+ phi|^2 re-solved at
    U(+-h): pins the factor 2 and the sign of -2 Re(Y^+ dD X)."""
    from oracle import hmc
    m0, csw = 0.1, 1.0
    U, rng = synth.gauge_field(DIMS, 0.3, 7)
    phi = synth.gaussian_spinor(DIMS, rng)
    A = orc.clover(DIMS, U, m0, csw)
    Y = hmc._solve(orc, DIMS, U, A, AP, phi, True, 1e-13)
    X = hmc._solve(orc, DIMS, U, A, AP, Y, False, 1e-13)
    F = hmc.fermion_force(orc, DIMS, U, A, AP, csw, X, Y)
    th = np.zeros((V, 4, 8))
    th[101, 3] = rng.standard_normal(8)
    h = 1e-5
    S = []
    for s in (+1, -1):
        Uh = _deform(U, th, s * h)
        Ah = orc.clover(DIMS, Uh, m0, csw)
        Yh = hmc._solve(orc, DIMS, Uh, Ah, AP, phi, True, 1e-13)
        S.append(np.vdot(Yh, Yh).real)
    fd = (S[0] - S[1]) / (2 * h)
    assert abs(fd - np.sum(F * th)) < 1e-6 * abs(fd)


@pytest.fixture(scope="module")
def traj_inputs():
    U, rng = synth.gauge_field(DIMS, 0.3, 11)
    pi = rng.standard_normal((V, 4, 8))
    eta = synth.gaussian_spinor(DIMS, rng)
    return U, pi, eta


def test_trajectory_is_reversible(orc, traj_inputs):
    from oracle import hmc
    U0, pi0, eta = traj_inputs
    args = dict(beta=5.5, m0=0.1, csw=1.0, bc=AP)
    U1, pi1, H0, H1, _ = hmc.trajectory(orc, DIMS, U0, pi0, eta, eps=0.05, nsteps=2, **args)
    # the pseudofermion stays the one drawn at U0: phi = D(U0)^+ eta; reverse
    # with that phi by passing eta' with D(U1)^+ eta' = phi
    A0 = orc.clover(DIMS, U0, args["m0"], args["csw"])
    phi = orc.apply_D(DIMS, U0, A0, AP, eta, dagger=True)
    A1 = orc.clover(DIMS, U1, args["m0"], args["csw"])
    eta1 = hmc._solve(orc, DIMS, U1, A1, AP, phi, True, 1e-14)
    U2, pi2, H0b, H1b, _ = hmc.trajectory(orc, DIMS, U1, -pi1, eta1, eps=0.05, nsteps=2, **args)
    assert rel(U2, U0) < 1e-10
    assert rel(-pi2, pi0) < 1e-9
    assert abs(H1b - H0) < 1e-8 * abs(H0)


def test_energy_violation_scales_with_step_squared(orc, traj_inputs):
    from oracle import hmc
    U0, pi0, eta = traj_inputs
    args = dict(beta=5.5, m0=0.1, csw=1.0, bc=AP)
    dH = []
    for eps, n in ((0.1, 1), (0.05, 2)):
        _, _, H0, H1, _ = hmc.trajectory(orc, DIMS, U0, pi0, eta, eps=eps, nsteps=n, **args)
        dH.append(H1 - H0)
    ratio = dH[0] / dH[1]
    assert 3.0 < ratio < 5.0, (dH, ratio)
