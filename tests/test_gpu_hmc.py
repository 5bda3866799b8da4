"""GPU HMC molecular dynamics (Sec. 1: the force the inversions feed) against
the oracle's trajectory: plaquette action, gauge force and link update
element by element, a complete leapfrog trajectory on 4^4 (links, momenta,
Hamiltonian), reversibility, and the second-order scaling of dH.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T


def _lat(dims, block, m0, csw, U):
    from paper_1109_4279_gb300 import binding
    lat = binding.Lattice(dims, block, m0, csw)
    lat.load_gauge(torch.from_numpy(U).cuda())
    return lat


def test_gauge_action_force_and_link_update_match_oracle():
    from oracle import hmc
    from paper_1109_4279_gb300 import binding
    dims, block = (8, 4, 4, 8), (2, 2, 2, 2)
    V = int(np.prod(dims))
    U, rng = synth.gauge_field(dims, 0.5, 13)
    lat = _lat(dims, block, 0.0, 1.0, U)
    Ut = torch.from_numpy(U).cuda()
    S = binding.qcd_gauge_action(lat.ctx, Ut, 5.5)
    assert abs(S - hmc.plaquette_action(U, dims, 5.5)) < 1e-11 * abs(S)
    F = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    binding.qcd_gauge_force(lat.ctx, Ut, 5.5, F)
    torch.cuda.synchronize()
    assert rel(F.cpu().numpy(), hmc.gauge_force(U, dims, 5.5)) < 1e-12
    pi = rng.standard_normal((V, 4, 8))
    binding.qcd_update_links(lat.ctx, Ut, torch.from_numpy(pi).cuda(), 0.3)
    torch.cuda.synchronize()
    Un = Ut.cpu().numpy()
    assert rel(Un, hmc.link_update(U, pi, 0.3)) < 1e-13
    UU = np.einsum("vmab,vmcb->vmac", Un, np.conj(Un))
    assert np.max(np.abs(UU - np.eye(3))) < 1e-13
    lat.close()


@pytest.fixture(scope="module")
def traj_case():
    dims = (4, 4, 4, 4)
    U, rng = synth.gauge_field(dims, 0.3, 11)
    pi = rng.standard_normal((256, 4, 8))
    eta = synth.gaussian_spinor(dims, rng)
    return dims, U, pi, eta


SP = dict(tol=1e-13, sap_prec="f64", nkv=16, max_restarts=200)


def test_trajectory_matches_oracle(orc, traj_case):
    from oracle import hmc
    dims, U, pi, eta = traj_case
    lat = _lat(dims, (2, 2, 2, 2), 0.1, 1.0, U)
    Ut, pit = torch.from_numpy(U.copy()).cuda(), torch.from_numpy(pi.copy()).cuda()
    info = lat.hmc_trajectory(Ut, pit, torch.from_numpy(eta).cuda(), 5.5, 0.05, 2, 0.0, **SP)
    U1, pi1, H0, H1, parts = hmc.trajectory(orc, dims, U, pi, eta, 5.5, 0.1, 1.0, AP, 0.05, 2)
    assert info["accepted"] == 1
    assert rel(Ut.cpu().numpy(), U1) < 1e-10
    assert rel(pit.cpu().numpy(), pi1) < 1e-9
    (k0, g0, f0), (k1, g1, f1) = parts
    for a, b in ((info["kin0"], k0), (info["S_g0"], g0), (info["S_f0"], f0), (info["kin1"], k1),
                 (info["S_g1"], g1), (info["S_f1"], f1)):
        assert abs(a - b) < 1e-10 * abs(b)
    assert abs(info["dH"] - (H1 - H0)) < 1e-8 * abs(H0)
    lat.close()


def test_trajectory_reversible(traj_case):
    """Forward, then backward from the end point with negated momenta and the
    same pseudofermion (eta' = D(U1)^-+ phi): the links return to U0."""
    from paper_1109_4279_gb300 import binding
    dims, U, pi, eta = traj_case
    lat = _lat(dims, (2, 2, 2, 2), 0.1, 1.0, U)
    Ut, pit, etat = torch.from_numpy(U.copy()).cuda(), torch.from_numpy(pi.copy()).cuda(), torch.from_numpy(eta).cuda()
    phi = torch.empty_like(etat)
    binding.qcd_apply_D(lat.ctx, etat, phi, dagger=True)       # phi = D(U0)^+ eta
    info = lat.hmc_trajectory(Ut, pit, etat, 5.5, 0.05, 2, 0.0, **SP)  # leaves U1 loaded
    eta1 = torch.zeros_like(etat)
    binding.qcd_solve_dagger(lat.ctx, phi, eta1, binding.solver_params(**SP))
    pit.neg_()
    info2 = lat.hmc_trajectory(Ut, pit, eta1, 5.5, 0.05, 2, 0.0, **SP)
    assert rel(Ut.cpu().numpy(), U) < 1e-10
    assert rel(-pit.cpu().numpy(), pi) < 1e-9
    assert abs(info2["H1"] - info["H0"]) < 1e-9 * abs(info["H0"])
    lat.close()


def test_dH_scales_with_step_squared():
    """Leapfrog is second order: at a fixed trajectory length, halving the
    step quarters dH once the step is small enough (on this 8^4 system dH =
    -20 eps^2 + 5300 eps^4 fits eps = 0.04, 0.02, 0.01 at trajectory length
    0.04 with every solver, so eps = 0.02 against 0.01 is in the asymptotic
    range)."""
    dims, block = (8, 8, 8, 8), (4, 4, 2, 2)
    U, rng = synth.gauge_field(dims, 0.3, 17)
    V = 8 ** 4
    pi = rng.standard_normal((V, 4, 8))
    eta = synth.gaussian_spinor(dims, rng)
    lat = _lat(dims, block, 0.1, 1.0, U)
    dH = []
    for eps, n in ((0.02, 2), (0.01, 4)):
        Ut, pit = torch.from_numpy(U.copy()).cuda(), torch.from_numpy(pi.copy()).cuda()
        info = lat.hmc_trajectory(Ut, pit, torch.from_numpy(eta).cuda(), 5.5, eps, n, 0.0, tol=1e-12, sap_prec="f32")
        dH.append(info["dH"])
    assert 3.0 < dH[0] / dH[1] < 5.0, dH
    lat.close()
