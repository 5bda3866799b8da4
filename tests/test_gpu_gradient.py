"""GPU gradient: force kernel, adjoint solve and autograd against the oracle
and finite differences (Sec. 1: the inversions feed the HMC fermion force).

Force convention: F_a(x, mu) = -Re(y^+ dD/dtheta_a x) for
U_mu(x) -> exp(i theta_a lambda_a / 2) U_mu(x); the oracle's dD/dh (pinned by
finite differences of D on the CPU) gives the same number per direction.
"""
import numpy as np
import pytest

from helpers import rel, vdot
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T


def _lattice(dims, block, U, m0, csw):
    from paper_1109_4279_gb300 import binding
    lat = binding.Lattice(dims, block, m0, csw)
    lat.load_gauge(torch.from_numpy(U).cuda())
    return lat


def _dU_single(U, site, mu, theta):
    dU = np.zeros_like(U)
    dU[site, mu] = 1j * synth.algebra(theta) @ U[site, mu]
    return dU


def test_force_all_links_4444(orc):
    """Every link and generator of a 4^4 lattice (random x, y): GPU force equals
    the oracle's -Re(y^+ dD x) direction by direction."""
    from paper_1109_4279_gb300 import binding
    dims, block, m0, csw = (4, 4, 4, 4), (2, 2, 2, 2), 0.1, 1.3
    U, rng = synth.gauge_field(dims, 0.5, 61)
    x = synth.gaussian_spinor(dims, rng)
    y = synth.gaussian_spinor(dims, rng)
    lat = _lattice(dims, block, U, m0, csw)
    F = torch.empty((lat.V, 4, 8), dtype=torch.float64, device="cuda")
    binding.qcd_force(lat.ctx, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), F)
    F = F.cpu().numpy()
    ref = np.empty_like(F)
    eye = np.eye(8)
    for s in range(lat.V):
        for mu in range(4):
            for a in range(8):
                d = orc.dD_apply(dims, U, _dU_single(U, s, mu, eye[a]), AP, csw, x)
                ref[s, mu, a] = -np.real(vdot(y, d))
    assert rel(F, ref) < 1e-12
    lat.close()


def _fd_directional(lat_dims, block, U, m0, csw, phi_t, x_t, th_field, h, sp):
    """Central finite difference of L = Re(phi^+ D(h)^-1 phi) along
    U -> exp(i h theta lambda / 2) U.  Each side solves only for the correction
    dx = D(h)^-1 (phi - D(h) x), so the solver tolerance applies to an O(h)
    quantity and the difference keeps its digits."""
    from paper_1109_4279_gb300 import binding
    vals = []
    for sgn in (+1, -1):
        Uh = np.einsum("vmab,vmbc->vmac", synth.su3_exp(sgn * h * synth.algebra(th_field)), U)
        lat = _lattice(lat_dims, block, Uh, m0, csw)
        Dx = lat.apply_D(x_t)
        r = phi_t - Dx
        dx = torch.zeros_like(r)
        binding.qcd_solve(lat.ctx, r, dx, 1, sp)
        vals.append(torch.real(torch.vdot(phi_t.flatten(), dx.flatten())).item())
        lat.close()
    return (vals[0] - vals[1]) / (2 * h)


def test_gradient_16x32_vs_oracle_and_fd(orc):
    """The 16^3 x 32 gradient workload: dL/dtheta along 32 random link
    directions (and one global direction) agrees with the oracle's directional
    derivative (same x, y) and with central finite differences (h = 1e-5) to
    1e-6 relative, |fd - g| <= 1e-6 |g| for every sampled direction;
    dL/dphi = x + y checks the adjoint solve."""
    from paper_1109_4279_gb300 import binding
    w = synth.WORKLOADS["16^3x32 gradient"]
    dims, block, m0, csw = w["dims"], w["block"], w["m0"], w["csw"]
    U, rng = synth.gauge_field(dims, w["eps"], w["seed"])
    phi = synth.gaussian_spinor(dims, rng)
    lat = _lattice(dims, block, U, m0, csw)
    V = lat.V
    phi_t = torch.from_numpy(phi).cuda()
    sp = binding.solver_params(tol=1e-12, sap_prec="f32")
    dphi = torch.empty_like(phi_t)
    F = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    x_t, y_t = torch.empty_like(phi_t), torch.empty_like(phi_t)
    binding.qcd_gradient(lat.ctx, phi_t, dphi, F, x_t, y_t, sp)
    x, y, F = x_t.cpu().numpy(), y_t.cpu().numpy(), F.cpu().numpy()
    assert rel(dphi.cpu().numpy(), x + y) < 1e-14
    A = orc.clover(dims, U, m0, csw)
    # x and y solve D x = phi and D^+ y = phi
    assert rel(orc.apply_D(dims, U, A, AP, x), phi) < 2e-12
    assert rel(orc.apply_D(dims, U, A, AP, y, dagger=True), phi) < 2e-12
    sites, mus, thetas = synth.link_directions(dims, 32, seed=5 + 1000)
    fd_sp = binding.solver_params(tol=1e-10, sap_prec="f32")
    for k, (s, mu, th) in enumerate(zip(sites, mus, thetas)):
        g = float(F[s, mu] @ th)
        o = -np.real(vdot(y, orc.dD_apply(dims, U, _dU_single(U, s, mu, th), AP, csw, x)))
        assert abs(g - o) <= 1e-10 * max(1.0, abs(o)), (k, g, o)
        if k < 8:  # finite differences: two extra solves each
            tf = np.zeros((V, 4, 8))
            tf[s, mu] = th
            fd = _fd_directional(dims, block, U, m0, csw, phi_t, x_t, tf, 1e-5, fd_sp)
            assert abs(fd - g) <= 1e-6 * abs(g), (k, fd, g)
    # one global direction over all links
    tf = np.random.default_rng(5 + 2000).standard_normal((V, 4, 8))
    g = float(np.sum(F * tf))
    fd = _fd_directional(dims, block, U, m0, csw, phi_t, x_t, tf, 1e-5, fd_sp)
    assert abs(fd - g) <= 1e-6 * abs(g), (fd, g)
    lat.close()


def test_autograd_matches_gradient(orc):
    """torch.autograd through DiracSolve: L = Re(phi^+ x) gives phi.grad = x + y
    and theta.grad = the force."""
    from paper_1109_4279_gb300 import autograd, binding
    dims, block, m0, csw = (8, 8, 8, 8), (4, 4, 4, 4), 0.0, 1.5
    U, rng = synth.gauge_field(dims, 0.5, 71)
    phi = synth.gaussian_spinor(dims, rng)
    lat = _lattice(dims, block, U, m0, csw)
    phi_t = torch.from_numpy(phi).cuda().requires_grad_(True)
    theta = torch.zeros((lat.V, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    x = autograd.dirac_solve(phi_t, theta, lat, tol=1e-12)
    L = torch.real(torch.sum(torch.conj(phi_t) * x))
    L.backward()
    sp = binding.solver_params(tol=1e-12)
    dphi = torch.empty_like(phi_t.detach())
    F = torch.empty_like(theta.detach())
    binding.qcd_gradient(lat.ctx, phi_t.detach(), dphi, F, None, None, sp)
    assert rel(phi_t.grad.cpu().numpy(), dphi.cpu().numpy()) < 1e-9
    assert rel(theta.grad.cpu().numpy(), F.cpu().numpy()) < 1e-9
    lat.close()
