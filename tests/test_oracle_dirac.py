"""Pins for the oracle's Dirac operator and clover term (CPU only).

Each test checks the oracle against something other than itself: the chiral
basis algebra, the free-field momentum-space closed form, gamma_5-hermiticity,
gauge covariance, hand-derived clover values for constant abelian fields, and
an independent dense numpy assembly of D (oracle/dense.py).
"""
import numpy as np
import pytest

from helpers import G, G5, rel, g5, vdot
from paper_1109_4279_gb300 import synth

AP = synth.ANTIPERIODIC_T


def _field(dims, eps, seed):
    U, rng = synth.gauge_field(dims, eps, seed)
    return U, rng


def test_chiral_basis():
    """The basis is Hermitian, Clifford, g5 = g0 g1 g2 g3 = diag(1,1,-1,-1),
    and sigma_{mu nu} is block diagonal (the clover splits into two 6x6 blocks)."""
    from oracle import dense
    gd = dense.gammas()
    for mu in range(4):
        assert np.allclose(G[mu], gd[mu])
        assert np.allclose(G[mu], G[mu].conj().T)
        for nu in range(4):
            ac = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))
            sig = 0.5j * (G[mu] @ G[nu] - G[nu] @ G[mu])
            assert np.allclose(sig[:2, 2:], 0) and np.allclose(sig[2:, :2], 0)
    assert np.allclose(G[0] @ G[1] @ G[2] @ G[3], G5)


@pytest.mark.parametrize("dims", [(4, 2, 4, 6), (6, 4, 2, 2)])
def test_free_field_plane_wave(orc, dims):
    """U = 1: a plane wave e^{ipx} u with antiperiodic p_0 = (2n+1)pi/T and
    p_k = 2 pi n_k / L_k is an eigenvector of the hopping stencil:
    D psi = [m0 + sum(1 - cos p) + i sum gamma_mu sin p_mu] psi (exactly)."""
    rng = np.random.default_rng(7)
    V = synth.volume(dims)
    U = synth.unit_gauge(dims)
    m0 = 0.137
    A = orc.clover(dims, U, m0, 1.7)   # F = 0 on the unit field: csw drops out
    x = np.array(np.unravel_index(np.arange(V), dims)).T
    for trial in range(3):
        n = rng.integers(0, 8, size=4)
        p = np.array([(2 * n[0] + 1) * np.pi / dims[0]] +
                     [2 * np.pi * n[k] / dims[k] for k in range(1, 4)])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (x @ p))
        psi = phase[:, None, None] * u[None]
        Mp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(np.sin(p[m]) * G[m] for m in range(4))
        expect = phase[:, None, None] * (Mp @ u)[None]
        out = orc.apply_D(dims, U, A, AP, psi)
        assert rel(out, expect) < 1e-13


def test_gamma5_hermiticity(orc):
    """(phi, g5 D g5 psi) = (D phi, psi) and the oracle's direct D^+ equals g5 D g5."""
    dims = (4, 4, 2, 6)
    U, rng = _field(dims, 0.5, 11)
    A = orc.clover(dims, U, -0.05, 1.5)
    phi = synth.gaussian_spinor(dims, rng)
    psi = synth.gaussian_spinor(dims, rng)
    lhs = vdot(phi, g5(orc.apply_D(dims, U, A, AP, g5(psi))))
    rhs = vdot(orc.apply_D(dims, U, A, AP, phi), psi)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13
    d_dag = orc.apply_D(dims, U, A, AP, psi, dagger=True)
    assert rel(d_dag, g5(orc.apply_D(dims, U, A, AP, g5(psi)))) < 1e-13


def test_clover_hermitian_and_chiral(orc):
    """A(x) is Hermitian and commutes with gamma_5 (block diagonal in chirality)."""
    dims = (4, 4, 4, 2)
    U, _ = _field(dims, 0.5, 12)
    A = orc.clover(dims, U, 0.0, 1.5)
    assert np.allclose(A, np.conj(np.swapaxes(A, 1, 2)), atol=1e-14)
    assert np.abs(A[:, :6, 6:]).max() < 1e-15 and np.abs(A[:, 6:, :6]).max() < 1e-15
    assert np.abs(A - 4.0 * np.eye(12)).max() > 1e-2  # the clover term is really there


def test_gauge_covariance(orc):
    """U_mu(x) -> L(x) U_mu(x) L(x+mu)^+, psi -> L psi gives D'(L psi) = L (D psi),
    with the clover rebuilt from the transformed links."""
    dims = (4, 2, 4, 4)
    U, rng = _field(dims, 0.5, 13)
    V = synth.volume(dims)
    Lam = synth.random_su3(V, rng)
    psi = synth.gaussian_spinor(dims, rng)
    shape = tuple(dims)
    Up = np.empty_like(U)
    Lr = Lam.reshape(shape + (3, 3))
    for mu in range(4):
        Lfwd = np.roll(Lr, -1, axis=mu).reshape(V, 3, 3)
        Up[:, mu] = Lam @ U[:, mu] @ np.conj(np.swapaxes(Lfwd, 1, 2))
    A = orc.clover(dims, U, 0.1, 1.3)
    Ap = orc.clover(dims, Up, 0.1, 1.3)
    out = orc.apply_D(dims, U, A, AP, psi)
    psi_p = np.einsum("vab,vsb->vsa", Lam, psi)
    out_p = orc.apply_D(dims, Up, Ap, AP, psi_p)
    assert rel(out_p, np.einsum("vab,vsb->vsa", Lam, out)) < 1e-13


@pytest.mark.parametrize("dims,bc", [((2, 2, 2, 2), AP), ((4, 2, 2, 2), AP), ((2, 2, 4, 2), (1, -1, 1, 1))])
def test_dense_assembly(orc, dims, bc):
    """The oracle's D, applied to every unit vector, equals the dense matrix built
    independently in numpy (oracle/dense.py)."""
    from oracle import dense
    U, _ = _field(dims, 0.7, 21)
    m0, csw = 0.1, 1.0
    V = synth.volume(dims)
    Dd = dense.dirac_matrix(dims, U, m0, csw, bc)
    A = orc.clover(dims, U, m0, csw)
    assert np.abs(A - dense.clover_blocks(dims, U, m0, csw)).max() < 1e-14
    E = np.eye(12 * V, dtype=complex).reshape(12 * V, V, 4, 3)
    cols = np.stack([orc.apply_D(dims, U, A, bc, E[k]).ravel() for k in range(12 * V)], axis=1)
    assert np.abs(cols - Dd).max() < 1e-13


def _abelian_links(dims, plane, theta, t):
    """Links equal to 1 except U_nu(x) = exp(i theta x_mu T), T = diag(t): a
    constant abelian field strength in the (mu, nu) plane."""
    mu, nu = plane
    V = synth.volume(dims)
    U = synth.unit_gauge(dims)
    x = np.array(np.unravel_index(np.arange(V), dims)).T
    ph = np.exp(1j * theta * np.outer(x[:, mu], t))
    U[:, nu] = 0
    for a in range(3):
        U[:, nu, a, a] = ph[:, a]
    return U


@pytest.mark.parametrize("plane,dims,spin_sign", [
    # sigma_12 = diag(-1, 1, -1, 1) in this basis, so the clover term is
    # -(csw/2) sigma_12 sin(theta T) = (csw/2) diag(1,-1,1,-1) x sin(theta T)
    ((1, 2), (4, 8, 4, 2), (1, -1, 1, -1)),
    # sigma_03 = diag(1, -1, -1, 1): clover = (csw/2) diag(-1, 1, 1, -1) x sin(theta T)
    ((0, 3), (8, 2, 2, 4), (-1, 1, 1, -1)),
])
def test_clover_abelian_closed_form(orc, plane, dims, spin_sign):
    """Constant abelian plaquette exp(i theta T) in one plane: every leaf equals
    it, Fhat = i sin(theta T), and the clover term is diagonal with the
    hand-derived values above.  T = diag(1, 1, -2) has sin(theta T) with a
    non-zero trace, which pins the reading "no trace subtraction"."""
    csw, m0 = 1.3, 0.2
    L_mu = dims[plane[0]]
    theta = 2 * np.pi / L_mu            # periodic in x_mu: theta * L_mu * t in 2 pi Z
    t = np.array([1.0, 1.0, -2.0])
    U = _abelian_links(dims, plane, theta, t)
    A = orc.clover(dims, U, m0, csw)
    diag = np.array([[4 + m0 + 0.5 * csw * s * np.sin(theta * ta) for ta in t] for s in spin_sign]).ravel()
    expect = np.broadcast_to(np.diag(diag), A.shape)
    assert np.abs(A - expect).max() < 1e-14
