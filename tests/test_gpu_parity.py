"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances are norm-wise relative over the whole field:
  operator D / D^+:  1e-12 (FP64), 1e-5 (FP32), 5e-3 (FP16 / BF16 storage);
  one SAP application: 1e-12 (FP64 block fields), 1e-5 (FP32), 5e-3 (16-bit);
  solves: true FP64 residual |b - D x| / |b| <= 1e-10, evaluated with the
  oracle's D, and |x - x_oracle| / |x_oracle| <= 1e-8 where the oracle solves.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T
TOL_D = {"f64": 1e-12, "f32": 1e-5, "f16": 5e-3, "bf16": 5e-3, "df64": 1e-12}


def _setup(dims, block, eps, seed, m0, csw, bc=AP):
    import oracle
    from paper_1109_4279_gb300 import binding
    U, rng = synth.gauge_field(dims, eps, seed)
    b = synth.gaussian_spinor(dims, rng)
    lat = binding.Lattice(dims, block, m0, csw, bc)
    lat.load_gauge(torch.from_numpy(U).cuda())
    A = oracle.clover(dims, U, m0, csw)
    return lat, U, A, b


CASES = [
    # dims, block, eps, seed, m0, csw, bc
    ((4, 4, 4, 4), (2, 2, 2, 2), 0.3, 1, 0.1, 1.0, AP),           # the 4^4 workload
    ((8, 4, 4, 8), (4, 2, 2, 4), 0.5, 7, -0.05, 1.5, AP),         # non-cubic blocks
    ((4, 8, 12, 4), (2, 4, 6, 2), 0.5, 8, 0.0, 1.2, (1, -1, 1, -1)),  # block extent 6, mixed signs
    ((32, 16, 16, 16), (4, 4, 4, 4), 0.5, 2, 0.0, 1.5, AP),       # the 16^3 x 32 workload
    ((16, 8, 8, 8), (8, 4, 4, 4), 0.5, 12, -0.05, 1.5, AP),       # the benchmarked block shape
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16", "df64"])
@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_parity(orc, case, prec, dagger):
    dims, block, eps, seed, m0, csw, bc = case
    lat, U, A, b = _setup(dims, block, eps, seed, m0, csw, bc)
    out = lat.apply_D(torch.from_numpy(b).cuda(), dagger=dagger, prec=prec).cpu().numpy()
    ref = orc.apply_D(dims, U, A, bc, b, dagger=dagger)
    assert rel(out, ref) < TOL_D[prec]
    lat.close()


def test_dirac_multi_rhs_and_free_field(orc):
    """Two right-hand sides in one call, and U = 1 (the clover term vanishes)."""
    from paper_1109_4279_gb300 import binding
    dims = (8, 4, 4, 4)
    U = synth.unit_gauge(dims)
    rng = np.random.default_rng(5)
    b = synth.gaussian_spinor(dims, rng, nrhs=2)
    lat = binding.Lattice(dims, (2, 2, 2, 2), 0.2, 1.7)
    lat.load_gauge(torch.from_numpy(U).cuda())
    out = lat.apply_D(torch.from_numpy(b).cuda()).cpu().numpy()
    A = orc.clover(dims, U, 0.2, 1.7)
    for k in range(2):
        assert rel(out[k], orc.apply_D(dims, U, A, AP, b[k])) < 1e-13
    lat.close()


def test_resident_field_apply(orc):
    """Import -> apply on resident fields -> export equals the oracle (FP32)."""
    from paper_1109_4279_gb300 import binding
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    lat, U, A, b = _setup(dims, block, 0.5, 3, -0.05, 1.5)
    fi = binding.qcd_field_create(lat.ctx, "f32")
    fo = binding.qcd_field_create(lat.ctx, "f32")
    bt = torch.from_numpy(b).cuda()
    binding.qcd_field_import(lat.ctx, fi, bt)
    binding.qcd_apply_D_field(lat.ctx, fi, fo)
    out = torch.empty_like(bt)
    binding.qcd_field_export(lat.ctx, fo, out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), orc.apply_D(dims, U, A, AP, b)) < 1e-5
    binding.qcd_field_free(fi)
    binding.qcd_field_free(fo)
    lat.close()


SAP_CASES = [
    ((4, 4, 4, 4), (2, 2, 2, 2), 0.3, 1, 0.1, 1.0),
    ((8, 8, 8, 8), (4, 4, 2, 2), 0.5, 9, 0.0, 1.5),
    ((8, 8, 8, 16), (4, 4, 4, 4), 0.5, 10, 0.0, 1.5),
    ((16, 8, 8, 8), (8, 4, 4, 4), 0.5, 12, -0.05, 1.5),   # the benchmarked block shape
]


@pytest.mark.parametrize("case", SAP_CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_sap_parity(orc, case, prec):
    dims, block, eps, seed, m0, csw = case
    vb = int(np.prod(block))
    if prec == "f64" and vb > 128:
        pytest.skip("FP64 block fields of a %d-site block exceed shared memory" % vb)
    if prec == "f32" and vb > 256:
        pytest.skip("FP32 block fields of a %d-site block exceed shared memory" % vb)
    lat, U, A, b = _setup(dims, block, eps, seed, m0, csw)
    psi = lat.sap(torch.from_numpy(b).cuda(), ncy=4, nmr=4, prec=prec).cpu().numpy()
    ref = orc.sap(dims, U, A, AP, block, b, ncy=4, nmr=4)
    assert rel(psi, ref) < {"f64": 1e-12, "f32": 1e-5, "f16": 5e-3, "bf16": 5e-3}[prec]
    lat.close()


def test_sap_single_cycle_and_deterministic(orc):
    """ncy = 1 (no incoming faces after the first half-sweep on black) and a
    bitwise repeat of the same call."""
    dims, block = (8, 8, 8, 8), (4, 4, 2, 2)
    lat, U, A, b = _setup(dims, block, 0.5, 11, 0.0, 1.5)
    bt = torch.from_numpy(b).cuda()
    p1 = lat.sap(bt, ncy=1, nmr=3, prec="f64").cpu().numpy()
    p2 = lat.sap(bt, ncy=1, nmr=3, prec="f64").cpu().numpy()
    assert np.array_equal(p1, p2)
    assert rel(p1, orc.sap(dims, U, A, AP, block, b, ncy=1, nmr=3)) < 1e-12
    lat.close()


def _oracle_residual(orc, dims, U, A, b, x):
    r = b - orc.apply_D(dims, U, A, AP, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("sap_prec,outer_prec", [("f64", "f64"), ("f32", "f64"), ("f16", "f64"), ("f64", "df64"),
                                                  ("f16", "df64")])
def test_solve_44_matches_oracle(orc, sap_prec, outer_prec):
    """The 4^4 workload: SAP (2^4 blocks, 4 MR steps, 4 cycles) + FGCR(16),
    with the FP64 or the double-float recursion."""
    w = synth.WORKLOADS["4^4 fp64"]
    dims = w["dims"]
    lat, U, A, b = _setup(dims, w["block"], w["eps"], w["seed"], w["m0"], w["csw"])
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, sap_prec=sap_prec, ncy=4, nmr=4, nkv=16,
                        outer_prec=outer_prec)
    x = x.cpu().numpy()
    assert info[0]["status"] == 0 and info[0]["true_residual"] <= 1e-10
    assert _oracle_residual(orc, dims, U, A, b, x) <= 1.05e-10
    x_or, *_ = orc.fgcr(dims, U, A, AP, b, nkv=16, tol=1e-12)
    assert rel(x, x_or) < 1e-8
    lat.close()


def test_solve_unpreconditioned_and_initial_guess(orc):
    w = synth.WORKLOADS["4^4 fp64"]
    dims = w["dims"]
    lat, U, A, b = _setup(dims, w["block"], w["eps"], w["seed"], w["m0"], w["csw"])
    bt = torch.from_numpy(b).cuda()
    x, info = lat.solve(bt, tol=1e-10, precond="none")
    assert info[0]["status"] == 0
    assert _oracle_residual(orc, dims, U, A, b, x.cpu().numpy()) <= 1.05e-10
    # restarting from the solution converges immediately
    x2, info2 = lat.solve(bt, x0=x, tol=1e-10)
    assert info2[0]["iterations"] == 0
    lat.close()


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "page-locked"])
def test_solve_host_pointers(orc, pinned):
    """b and x in host memory (pageable or page-locked): the library stages
    them through device memory; the solution is bit for bit the one of the
    same solve on device buffers."""
    w = synth.WORKLOADS["4^4 fp64"]
    dims = w["dims"]
    lat, U, A, b = _setup(dims, w["block"], w["eps"], w["seed"], w["m0"], w["csw"])
    from paper_1109_4279_gb300 import binding
    bt = torch.from_numpy(b.copy())
    x = torch.zeros_like(bt)
    if pinned:
        bt, x = bt.pin_memory(), x.pin_memory()
    st, info = binding.qcd_solve(lat.ctx, bt, x, 1, binding.solver_params(tol=1e-10))
    assert st == 0
    assert _oracle_residual(orc, dims, U, A, b, x.numpy()) <= 1.05e-10
    xd = torch.zeros_like(bt).cuda()
    binding.qcd_solve(lat.ctx, bt.cuda(), xd, 1, binding.solver_params(tol=1e-10))
    assert torch.equal(xd.cpu(), x)
    lat.close()


@pytest.fixture(scope="module")
def solved_16x32(orc):
    """The 16^3 x 32 workload and the oracle's solution of it (unpreconditioned
    FP64 GCR(16) to |b - D x| / |b| <= 1e-12)."""
    w = synth.WORKLOADS["16^3x32 fp32"]
    dims = w["dims"]
    U, rng = synth.gauge_field(dims, w["eps"], w["seed"])
    b = synth.gaussian_spinor(dims, rng)
    A = orc.clover(dims, U, w["m0"], w["csw"])
    x_or, _, _, conv, res = orc.fgcr(dims, U, A, AP, b, nkv=16, tol=1e-12, max_restarts=400)
    assert conv and res <= 1e-12
    return w, U, A, b, x_or


@pytest.mark.parametrize("sap_prec", ["f32", "f16", "bf16"])
def test_solve_16x32(orc, solved_16x32, sap_prec):
    """The 16^3 x 32 workload (4^4 blocks, FP64 recursion) with each block-field
    precision: the GPU solution's true residual, recomputed with the oracle's
    operator, is below 1e-10, and the solution agrees with the oracle's
    solution to 1e-8 (two solutions with residuals 1e-10 and 1e-12 differ by
    at most cond(D) 1.01e-10; on this lattice the gap between the oracle's own
    1e-10 and 1e-12 solutions is 6e-10)."""
    w, U, A, b, x_or = solved_16x32
    dims = w["dims"]
    from paper_1109_4279_gb300 import binding
    lat = binding.Lattice(dims, w["block"], w["m0"], w["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, sap_prec=sap_prec)
    assert info[0]["status"] == 0, info
    x = x.cpu().numpy()
    assert _oracle_residual(orc, dims, U, A, b, x) <= 1.05e-10
    assert rel(x, x_or) < 1e-8
    lat.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_resident_field_multi_rhs(orc, prec):
    """Three right-hand sides in one resident field, one operator launch for
    all three: each equals the oracle's D applied to it."""
    from paper_1109_4279_gb300 import binding
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    lat, U, A, _ = _setup(dims, block, 0.5, 11, -0.05, 1.5)
    rng = np.random.default_rng(12)
    b = synth.gaussian_spinor(dims, rng, nrhs=3)
    fi = binding.qcd_field_create_n(lat.ctx, prec, 3)
    fo = binding.qcd_field_create_n(lat.ctx, prec, 3)
    bt = torch.from_numpy(b).cuda()
    binding.qcd_field_import(lat.ctx, fi, bt)
    binding.qcd_apply_D_field(lat.ctx, fi, fo)
    out = torch.empty_like(bt)
    binding.qcd_field_export(lat.ctx, fo, out)
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    for k in range(3):
        assert rel(out[k], orc.apply_D(dims, U, A, AP, b[k])) < TOL_D[prec]
    binding.qcd_field_free(fi)
    binding.qcd_field_free(fo)
    lat.close()


@pytest.mark.parametrize("sap_prec,residual_prec", [("f16", "df64"), ("bf16", "df64"), ("f16", "f64")])
def test_solve_16x32_df64_recursion(orc, solved_16x32, sap_prec, residual_prec):
    """The double-float recursion (chi = D phi, Gram-Schmidt, dots and updates
    on pairs of FP32 values, FP64 solution), with the restart residual's D x
    in double-float arithmetic (the default) or in FP64: true residual below
    1e-10, the reported residual equal to the oracle's recomputed one, the
    oracle's solution to 1e-8 and the FP64 recursion's iteration count."""
    w, U, A, b, x_or = solved_16x32
    dims = w["dims"]
    from paper_1109_4279_gb300 import binding
    lat = binding.Lattice(dims, w["block"], w["m0"], w["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, sap_prec=sap_prec, outer_prec="df64",
                        residual_prec=residual_prec)
    assert info[0]["status"] == 0, info
    x = x.cpu().numpy()
    res = _oracle_residual(orc, dims, U, A, b, x)
    assert res <= 1.05e-10
    assert abs(res - info[0]["true_residual"]) < 1e-13
    assert rel(x, x_or) < 1e-8
    _, info64 = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, sap_prec=sap_prec, outer_prec="f64")
    assert abs(info64[0]["iterations"] - info[0]["iterations"]) <= 1
    lat.close()


def test_solve_outer_f32_split(orc, solved_16x32):
    """The split of Sec. 4: chi_k = D phi_k in FP32 inside the Krylov
    recursion, the residual recomputed in FP64 at every restart; the FP64
    true residual still reaches 1e-10 and the solution agrees with the
    oracle's to 1e-8."""
    w, U, A, b, x_or = solved_16x32
    dims = w["dims"]
    from paper_1109_4279_gb300 import binding
    lat = binding.Lattice(dims, w["block"], w["m0"], w["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, sap_prec="f16", outer_prec="f32")
    assert info[0]["status"] == 0, info
    x = x.cpu().numpy()
    assert _oracle_residual(orc, dims, U, A, b, x) <= 1.05e-10
    assert rel(x, x_or) < 1e-8
    lat.close()


@pytest.mark.parametrize("precond", ["sap", "none"])
def test_solve_outer_f32_small(orc, precond):
    """FP32 recursion with FP64 restarts on 8^4 (2 x 2 x 4 x 4 blocks): the
    solution's FP64 residual, recomputed by the oracle, reaches 1e-10, and
    the solution agrees with the all-FP64 recursion's."""
    dims, block = (8, 8, 8, 8), (4, 4, 2, 2)
    lat, U, A, b = _setup(dims, block, 0.5, 9, 0.0, 1.5)
    bt = torch.from_numpy(b).cuda()
    x32, info = lat.solve(bt, tol=1e-10, precond=precond, sap_prec="f32", outer_prec="f32", max_restarts=400)
    assert info[0]["status"] == 0, info
    assert _oracle_residual(orc, dims, U, A, b, x32.cpu().numpy()) <= 1.05e-10
    x64, _ = lat.solve(bt, tol=1e-12, precond=precond, sap_prec="f32", outer_prec="f64", max_restarts=400)
    # both residuals <= 1e-10 |b|: the solutions differ by at most
    # |D^-1| |D| 2e-10 relative, well below 1e-7 for this mass
    assert rel(x32.cpu().numpy(), x64.cpu().numpy()) < 1e-7
    lat.close()
