"""GPU CG on the normal equations (the CG fallback of Sec. 4) against the
oracle: the same iteration on D^+ D in FP64, solutions equal to dense LU /
the oracle's CGNE, and the automatic switch from a stagnating FGCR.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T


def _setup(dims, block, eps, seed, m0, csw):
    import oracle
    from paper_1109_4279_gb300 import binding
    U, rng = synth.gauge_field(dims, eps, seed)
    b = synth.gaussian_spinor(dims, rng)
    lat = binding.Lattice(dims, block, m0, csw)
    lat.load_gauge(torch.from_numpy(U).cuda())
    A = oracle.clover(dims, U, m0, csw)
    return lat, U, A, b


def _res(orc, dims, U, A, b, x):
    return np.linalg.norm(b - orc.apply_D(dims, U, A, AP, x)) / np.linalg.norm(b)


def test_cg_matches_oracle_cgne(orc):
    """8^4 at m0 = -0.2: the GPU's iteration count is the oracle's rounded up
    to its 16-iteration residual check, and the solutions agree."""
    from oracle.cgne import cgne
    dims, block = (8, 8, 8, 8), (4, 4, 2, 2)
    lat, U, A, b = _setup(dims, block, 0.5, 21, -0.2, 1.5)
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, solver="cg")
    assert info[0]["status"] == 0, info
    x = x.cpu().numpy()
    assert _res(orc, dims, U, A, b, x) <= 1.05e-10
    D = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape)).ravel()
    Dh = lambda v: orc.apply_D(dims, U, A, AP, v.reshape(b.shape), dagger=True).ravel()
    xo, io = cgne(D, Dh, b, tol=1e-10, max_iter=5000)
    assert io["converged"]
    assert io["iterations"] <= info[0]["cg_iterations"] <= io["iterations"] + 16 + 2
    assert rel(x.ravel(), xo) < 1e-8
    lat.close()


def test_cg_44_matches_dense_lu(orc):
    from oracle import dense
    w = synth.WORKLOADS["4^4 fp64"]
    dims = w["dims"]
    lat, U, A, b = _setup(dims, w["block"], w["eps"], w["seed"], w["m0"], w["csw"])
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-12, solver="cg")
    assert info[0]["status"] == 0, info
    D = dense.dirac_matrix(dims, U, w["m0"], w["csw"], AP)
    assert rel(x.cpu().numpy().ravel(), np.linalg.solve(D, b.ravel())) < 1e-10
    lat.close()


def test_fgcr_falls_back_to_cg(orc):
    """FGCR with 2 Krylov vectors and one restart cannot reach 1e-10 on
    16^3 x 32: alone it reports not-converged; with cg_fallback the solve
    continues from its iterate with CG and converges."""
    from paper_1109_4279_gb300 import binding
    w = synth.WORKLOADS["16^3x32 fp32"]
    dims = w["dims"]
    lat, U, A, b = _setup(dims, w["block"], w["eps"], w["seed"], w["m0"], w["csw"])
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    st, info = binding.qcd_solve(lat.ctx, bt, x, 1,
                                 binding.solver_params(tol=1e-10, nkv=2, max_restarts=1, sap_prec="f16"),
                                 raise_on_fail=False)
    assert st != 0 and info[0]["cg_iterations"] == 0
    x, info = lat.solve(bt, tol=1e-10, nkv=2, max_restarts=1, sap_prec="f16", cg_fallback=1)
    assert info[0]["status"] == 0, info
    assert info[0]["iterations"] == 2 and info[0]["cg_iterations"] > 0
    assert _res(orc, dims, U, A, b, x.cpu().numpy()) <= 1.05e-10
    lat.close()


def test_cg_eo_matches_oracle(orc):
    """Even/odd-preconditioned CG on 8^4 at m0 = -0.2: the iteration count is
    the oracle's (cg_eo) rounded up to the 16-iteration residual check, the
    solution agrees, and it needs fewer iterations than CG on D^+ D."""
    from oracle import eo
    dims, block = (8, 8, 8, 8), (4, 4, 2, 2)
    lat, U, A, b = _setup(dims, block, 0.5, 21, -0.2, 1.5)
    bt = torch.from_numpy(b).cuda()
    x, info = lat.solve(bt, tol=1e-10, solver="cg_eo")
    assert info[0]["status"] == 0, info
    x = x.cpu().numpy()
    assert _res(orc, dims, U, A, b, x) <= 1.05e-10
    xo, io = eo.cg_eo(orc, dims, U, A, AP, b, tol=1e-10)
    assert io["converged"]
    assert io["iterations"] <= info[0]["cg_iterations"] <= io["iterations"] + 16 + 2
    assert rel(x, xo) < 1e-8
    _, info_ne = lat.solve(bt, tol=1e-10, solver="cg")
    assert info[0]["cg_iterations"] < info_ne[0]["cg_iterations"]
    lat.close()


def test_cg_eo_44_dense_lu_and_adjoint(orc):
    """4^4: the even/odd CG solution equals dense LU, for D and (through
    qcd_solve_dagger) for D^+."""
    from oracle import dense
    from paper_1109_4279_gb300 import binding
    w = synth.WORKLOADS["4^4 fp64"]
    dims = w["dims"]
    lat, U, A, b = _setup(dims, w["block"], w["eps"], w["seed"], w["m0"], w["csw"])
    D = dense.dirac_matrix(dims, U, w["m0"], w["csw"], AP)
    bt = torch.from_numpy(b).cuda()
    x, info = lat.solve(bt, tol=1e-12, solver="cg_eo")
    assert info[0]["status"] == 0, info
    assert rel(x.cpu().numpy().ravel(), np.linalg.solve(D, b.ravel())) < 1e-10
    y = torch.zeros_like(bt)
    st, inf = binding.qcd_solve_dagger(lat.ctx, bt, y, binding.solver_params(tol=1e-12, solver="cg_eo"))
    assert st == 0 and inf["cg_iterations"] > 0
    assert rel(y.cpu().numpy().ravel(), np.linalg.solve(D.conj().T, b.ravel())) < 1e-10
    lat.close()


def test_fgcr_falls_back_to_cg_eo(orc):
    """cg_fallback = 2 continues a failed FGCR with the even/odd CG."""
    from paper_1109_4279_gb300 import binding
    w = synth.WORKLOADS["16^3x32 fp32"]
    dims = w["dims"]
    lat, U, A, b = _setup(dims, w["block"], w["eps"], w["seed"], w["m0"], w["csw"])
    bt = torch.from_numpy(b).cuda()
    x, info = lat.solve(bt, tol=1e-10, nkv=2, max_restarts=1, sap_prec="f16", cg_fallback=2)
    assert info[0]["status"] == 0, info
    assert info[0]["iterations"] == 2 and info[0]["cg_iterations"] > 0
    assert _res(orc, dims, U, A, b, x.cpu().numpy()) <= 1.05e-10
    for kw in (dict(solver=4), dict(cg_fallback=3)):
        xx = torch.zeros_like(bt)
        st, _ = binding.qcd_solve(lat.ctx, bt, xx, 1, binding.solver_params(tol=1e-10, **kw), raise_on_fail=False)
        assert st == -1, kw
    lat.close()
