"""Pins for the oracle's SAP preconditioner, MR block solver and (F)GCR (CPU).

References: SAP cycle and MR block solves (Sec. 4), even/odd split inside
blocks (Sec. 5, Table 1), FGCR with restarts (Sec. 4).  The checks use dense
numpy algebra assembled independently (oracle/dense.py).
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

AP = synth.ANTIPERIODIC_T


@pytest.fixture(scope="module")
def lat44():
    """The 4^4 workload: eps = 0.3, seed 1, m0 = 0.1, csw = 1.0, 2^4 blocks."""
    import oracle
    from oracle import dense
    w = synth.WORKLOADS["4^4 fp64"]
    dims = w["dims"]
    U, rng = synth.gauge_field(dims, w["eps"], w["seed"])
    b = synth.gaussian_spinor(dims, rng)
    A = oracle.clover(dims, U, w["m0"], w["csw"])
    D = dense.dirac_matrix(dims, U, w["m0"], w["csw"], AP)
    return dict(dims=dims, U=U, A=A, D=D, b=b, w=w)


def _blocks(orc, dims, block):
    nb = [dims[m] // block[m] for m in range(4)]
    out = []
    for n in range(int(np.prod(nb))):
        c = np.unravel_index(n, nb)
        out.append((orc.block_sites(dims, block, n), int(sum(c)) % 2))
    return out


def _dofs(sites):
    return (12 * sites[:, None] + np.arange(12)[None, :]).ravel()


def test_sap_exact_block_solves_closed_form(orc, lat44):
    """With converged block solves one SAP cycle is
    M = K_w + K_b - K_b D K_w,  K_c = (+)_{blocks of colour c} D_blk^-1,
    and after the black half-sweep the residual vanishes on black blocks."""
    dims, U, A, D, b = lat44["dims"], lat44["U"], lat44["A"], lat44["D"], lat44["b"]
    block = (2, 2, 2, 2)
    eta = b.ravel()

    def K(colour, v):
        out = np.zeros_like(v)
        for sites, col in _blocks(orc, dims, block):
            if col != colour:
                continue
            d = _dofs(sites)
            out[d] = np.linalg.solve(D[np.ix_(d, d)], v[d])
        return out

    kw = K(0, eta)
    expect = kw + K(1, eta - D @ kw)
    for eo in (True, False):
        psi, rho = orc.sap(dims, U, A, AP, block, b, ncy=1, nmr=300, eo=eo, return_rho=True)
        assert rel(psi.ravel(), expect) < 1e-11
        assert rel(rho.ravel(), eta - D @ psi.ravel()) < 1e-12   # rho tracks eta - D psi
        for sites, col in _blocks(orc, dims, block):
            if col == 1:
                assert np.linalg.norm(rho.ravel()[_dofs(sites)]) < 1e-10 * np.linalg.norm(eta)


def test_sap_multiple_cycles_are_iterative_refinement(orc, lat44):
    """n_cy cycles with exact block solves: psi_{n} = psi_{n-1} + M_1 (eta - D psi_{n-1})."""
    dims, U, A, D, b = lat44["dims"], lat44["U"], lat44["A"], lat44["D"], lat44["b"]
    block = (2, 2, 2, 2)
    psi1 = orc.sap(dims, U, A, AP, block, b, ncy=1, nmr=300).ravel()
    r1 = (b.ravel() - D @ psi1).reshape(b.shape)
    psi2 = orc.sap(dims, U, A, AP, block, b, ncy=2, nmr=300).ravel()
    assert rel(psi2, psi1 + orc.sap(dims, U, A, AP, block, r1, ncy=1, nmr=300).ravel()) < 1e-11


def test_sap_block_order_independent(orc, lat44):
    """Blocks of one colour are independent: visiting them in reverse order
    changes only the rounding of the residual sums."""
    dims, U, A, b = lat44["dims"], lat44["U"], lat44["A"], lat44["b"]
    p1 = orc.sap(dims, U, A, AP, (2, 2, 2, 2), b, ncy=3, nmr=4)
    p2 = orc.sap(dims, U, A, AP, (2, 2, 2, 2), b, ncy=3, nmr=4, reverse=True)
    assert rel(p1, p2) < 1e-14


def test_sap_rejects_odd_block_counts(orc, lat44):
    dims, U, A, b = lat44["dims"], lat44["U"], lat44["A"], lat44["b"]
    with pytest.raises(RuntimeError):
        orc.sap(dims, U, A, AP, (4, 2, 2, 2), b, ncy=1, nmr=1)  # 1 block along t


def _schur(D, sites, dims):
    """Dense D_blk split by global site parity."""
    V = synth.volume(dims)
    x = np.array(np.unravel_index(sites, dims)).T
    par = x.sum(axis=1) % 2
    d = _dofs(sites)
    Db = D[np.ix_(d, d)]
    e = np.concatenate([np.arange(12 * k, 12 * k + 12) for k in np.where(par == 0)[0]])
    o = np.concatenate([np.arange(12 * k, 12 * k + 12) for k in np.where(par == 1)[0]])
    return Db, e, o


def test_block_mr_invariants(orc, lat44):
    """EO-MR on one block: the block residual vanishes on odd sites, is
    non-increasing in n_mr, the first step's residual is orthogonal to
    Dhat etahat (optimal alpha), and many steps converge to D_blk^-1 rho."""
    dims, U, A, D = lat44["dims"], lat44["U"], lat44["A"], lat44["D"]
    block = (2, 2, 2, 2)
    rng = np.random.default_rng(3)
    n = 5
    sites = orc.block_sites(dims, block, n)
    Db, e, o = _schur(D, sites, dims)
    rho = rng.standard_normal((16, 4, 3)) + 1j * rng.standard_normal((16, 4, 3))
    r = rho.ravel()
    Aoo_inv = np.linalg.inv(Db[np.ix_(o, o)])
    Dhat = Db[np.ix_(e, e)] - Db[np.ix_(e, o)] @ Aoo_inv @ Db[np.ix_(o, e)]
    etahat = r[e] - Db[np.ix_(e, o)] @ Aoo_inv @ r[o]
    last = np.inf
    for nmr in range(0, 7):
        chi = orc.block_mr(dims, U, A, AP, block, n, rho, nmr).ravel()
        res = r - Db @ chi
        assert np.linalg.norm(res[o]) < 1e-13 * np.linalg.norm(r)
        nr = np.linalg.norm(res)
        assert nr <= last * (1 + 1e-14)
        last = nr
        if nmr == 1:
            assert abs(np.vdot(Dhat @ etahat, res[e])) < 1e-12 * np.linalg.norm(etahat) ** 2
    chi = orc.block_mr(dims, U, A, AP, block, n, rho, 300).ravel()
    assert rel(chi, np.linalg.solve(Db, r)) < 1e-12
    # plain (non-EO) MR converges to the same block solution
    chi = orc.block_mr(dims, U, A, AP, block, n, rho, 400, eo=False).ravel()
    assert rel(chi, np.linalg.solve(Db, r)) < 1e-10


def test_gcr_matches_dense_lu_2444(orc):
    """Unpreconditioned GCR on the 2^4 copy of the 4^4 workload (fresh seed-1
    generator) reaches the LU solution."""
    from oracle import dense
    w = synth.WORKLOADS["4^4 fp64"]
    dims = (2, 2, 2, 2)
    U, rng = synth.gauge_field(dims, w["eps"], w["seed"])
    b = synth.gaussian_spinor(dims, rng)
    A = orc.clover(dims, U, w["m0"], w["csw"])
    D = dense.dirac_matrix(dims, U, w["m0"], w["csw"], AP)
    x_lu = np.linalg.solve(D, b.ravel())
    x, iters, cycles, conv, res = orc.fgcr(dims, U, A, AP, b, nkv=16, tol=1e-12)
    assert conv and res <= 1e-12
    assert np.linalg.norm(b.ravel() - D @ x.ravel()) / np.linalg.norm(b) <= 1.01e-12
    assert rel(x.ravel(), x_lu) < 1e-10


def test_gcr_cycle_is_krylov_least_squares(orc):
    """One GCR cycle of k steps from x0 = 0 returns the minimiser of
    |b - D x| over the Krylov space span{b, Db, ..., D^{k-1} b}: this pins the
    Gram-Schmidt coefficients and the triangular back-substitution."""
    from oracle import dense
    dims = (2, 2, 2, 2)
    U, rng = synth.gauge_field(dims, 0.4, 99)
    b = synth.gaussian_spinor(dims, rng)
    A = orc.clover(dims, U, 0.3, 1.0)
    D = dense.dirac_matrix(dims, U, 0.3, 1.0, AP)
    k = 5
    x, iters, cycles, conv, res = orc.fgcr(dims, U, A, AP, b, nkv=k, max_restarts=1, tol=1e-30)
    assert iters == k and cycles == 1
    K = [b.ravel()]
    for _ in range(k - 1):
        K.append(D @ K[-1])
    K = np.stack(K, axis=1)
    Q, _ = np.linalg.qr(K)
    coef, *_ = np.linalg.lstsq(D @ Q, b.ravel(), rcond=None)
    assert rel(x.ravel(), Q @ coef) < 1e-9


def test_fgcr_sap_matches_dense_lu_44(orc, lat44):
    """SAP-preconditioned FGCR (2^4 blocks, 4 MR steps, 4 cycles, restart 16)
    on the 4^4 workload converges to the dense LU solution."""
    dims, U, A, D, b = lat44["dims"], lat44["U"], lat44["A"], lat44["D"], lat44["b"]
    x_lu = np.linalg.solve(D, b.ravel())
    x, iters, cycles, conv, res = orc.fgcr(dims, U, A, AP, b, nkv=16, tol=1e-12, precond=True,
                                           block=(2, 2, 2, 2), ncy=4, nmr=4)
    assert conv and res <= 1e-12
    assert rel(x.ravel(), x_lu) < 1e-10
    # the preconditioner must pay off against plain GCR
    _, it_plain, *_ = orc.fgcr(dims, U, A, AP, b, nkv=16, tol=1e-12)
    assert iters < it_plain
