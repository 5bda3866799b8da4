"""Edge cases of the GPU path: degenerate right-hand sides, invalid inputs,
unsupported shapes at the size limits, ragged lattices, exhausted restarts
and run-to-run determinism.  Every error comes back as a status code; none
faults or hangs the device.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T


def _lat(dims, block, m0=0.0, csw=1.5, eps=0.5, seed=3):
    from paper_1109_4279_gb300 import binding
    U, rng = synth.gauge_field(dims, eps, seed)
    lat = binding.Lattice(dims, block, m0, csw)
    lat.load_gauge(torch.from_numpy(U).cuda())
    return lat, U, rng


def test_zero_rhs_gives_zero_solution():
    lat, U, rng = _lat((8, 8, 8, 8), (4, 4, 2, 2))
    b = torch.zeros((8 ** 4, 4, 3), dtype=torch.complex128, device="cuda")
    x0 = torch.ones_like(b)
    x, info = lat.solve(b, x0=x0, tol=1e-10, sap_prec="f16")
    assert info[0]["status"] == 0 and info[0]["iterations"] == 0
    assert torch.count_nonzero(x).item() == 0
    lat.close()


def test_zero_rhs_inside_a_batch(orc):
    """nrhs = 3 with the middle right-hand side zero: it returns x = 0 and the
    other two converge."""
    dims = (8, 8, 8, 8)
    lat, U, rng = _lat(dims, (4, 4, 2, 2))
    b = synth.gaussian_spinor(dims, rng, nrhs=3)
    b[1] = 0
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, sap_prec="f16")
    assert [i["status"] for i in info] == [0, 0, 0]
    x = x.cpu().numpy()
    assert np.count_nonzero(x[1]) == 0
    A = orc.clover(dims, U, 0.0, 1.5)
    for k in (0, 2):
        assert np.linalg.norm(b[k] - orc.apply_D(dims, U, A, AP, x[k])) <= 1.05e-10 * np.linalg.norm(b[k])
    lat.close()


def test_nan_input_is_reported_not_hung():
    from paper_1109_4279_gb300 import binding
    dims = (8, 8, 8, 8)
    lat, U, rng = _lat(dims, (4, 4, 2, 2))
    b = torch.from_numpy(synth.gaussian_spinor(dims, rng)).cuda()
    b[17, 2, 1] = complex(float("nan"), 0.0)
    x = torch.zeros_like(b)
    st, info = binding.qcd_solve(lat.ctx, b, x, 1, binding.solver_params(tol=1e-10), raise_on_fail=False)
    assert st == -10 and info[0]["status"] == -10  # QCD_NAN
    lat.close()


def test_non_su3_links_are_rejected():
    from paper_1109_4279_gb300 import binding
    dims = (8, 8, 8, 8)
    U, _ = synth.gauge_field(dims, 0.5, 3)
    U[100, 2] *= 1.001
    h = binding.qcd_create(dims, (4, 4, 2, 2), 0.0, 1.5)
    with pytest.raises(binding.QcdError) as e:
        binding.qcd_load_gauge(h, torch.from_numpy(U).cuda())
    assert e.value.status == -6  # QCD_ERR_NOT_SU3
    binding.qcd_destroy(h)


def test_solve_before_gauge_is_a_state_error():
    from paper_1109_4279_gb300 import binding
    h = binding.qcd_create((8, 8, 8, 8), (4, 4, 2, 2), 0.0, 1.5)
    b = torch.ones((8 ** 4, 4, 3), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(b)
    st, _ = binding.qcd_solve(h, b, x, 1, binding.solver_params(), raise_on_fail=False)
    assert st == -5  # QCD_ERR_STATE
    binding.qcd_destroy(h)


def test_size_limits_of_the_sap_kernel():
    """Vb = 1024 (8x8x4x4 blocks) exceeds the SAP kernel's block size: the solve
    reports QCD_ERR_UNSUPPORTED, and the same lattice solves without the
    preconditioner; FP32 block fields of 8x4x4x4 blocks do not fit in shared
    memory (unsupported) while FP16 ones do."""
    from paper_1109_4279_gb300 import binding
    dims = (16, 16, 8, 8)
    lat, U, rng = _lat(dims, (8, 8, 4, 4))
    b = torch.from_numpy(synth.gaussian_spinor(dims, rng)).cuda()
    x = torch.zeros_like(b)
    st, _ = binding.qcd_solve(lat.ctx, b, x, 1, binding.solver_params(tol=1e-10), raise_on_fail=False)
    assert st == -11
    x, info = lat.solve(b, tol=1e-10, precond="none", max_restarts=400)
    assert info[0]["status"] == 0
    lat.close()
    lat, U, rng = _lat(dims, (8, 4, 4, 4))
    x = torch.zeros_like(b)
    st, _ = binding.qcd_solve(lat.ctx, b, x, 1, binding.solver_params(tol=1e-10, sap_prec="f32"), raise_on_fail=False)
    assert st == -11
    x, info = lat.solve(b, tol=1e-10, sap_prec="f16")
    assert info[0]["status"] == 0
    lat.close()


def test_bad_solver_parameters():
    from paper_1109_4279_gb300 import binding
    lat, U, rng = _lat((8, 8, 8, 8), (4, 4, 2, 2))
    b = torch.from_numpy(synth.gaussian_spinor((8, 8, 8, 8), rng)).cuda()
    for kw in (dict(tol=0.0), dict(nkv=0), dict(nkv=65), dict(ncy=0), dict(sap_prec=7),
               dict(outer_prec="f32", inner_tol=1.5), dict(outer_prec="df64", residual_prec="f32")):
        x = torch.zeros_like(b)
        st, _ = binding.qcd_solve(lat.ctx, b, x, 1, binding.solver_params(**kw), raise_on_fail=False)
        assert st == -1, kw
    lat.close()


def test_df64_recursion_with_and_without_preconditioner(orc):
    """The double-float recursion keeps phi_k in FP32 behind the SAP (its
    output is FP32-exact) and in double-float without a preconditioner (phi_k =
    rho_k); the same workspace switches between the two.  Every solve meets the
    oracle's residual, and the SAP solve after the switch repeats the first."""
    dims = (8, 8, 8, 8)
    lat, U, rng = _lat(dims, (4, 4, 4, 4))
    bn = synth.gaussian_spinor(dims, rng)
    b = torch.from_numpy(bn).cuda()
    A = orc.clover(dims, U, 0.0, 1.5)
    runs = []
    for precond in ("sap", "none", "sap"):
        x, info = lat.solve(b, tol=1e-10, precond=precond, sap_prec="f16", outer_prec="df64", max_restarts=200)
        assert info[0]["status"] == 0, (precond, info)
        xn = x.cpu().numpy()
        res = np.linalg.norm(bn - orc.apply_D(dims, U, A, AP, xn)) / np.linalg.norm(bn)
        assert res <= 1.05e-10 and abs(res - info[0]["true_residual"]) < 1e-13, precond
        runs.append((xn, info[0]["iterations"]))
    assert runs[2][1] == runs[0][1] and np.array_equal(runs[2][0], runs[0][0])
    assert runs[1][1] > runs[0][1]  # the unpreconditioned recursion takes more iterations
    lat.close()


def test_exhausted_restarts_return_the_best_iterate(orc):
    from paper_1109_4279_gb300 import binding
    dims = (8, 8, 8, 8)
    lat, U, rng = _lat(dims, (4, 4, 2, 2))
    bn = synth.gaussian_spinor(dims, rng)
    b = torch.from_numpy(bn).cuda()
    x = torch.zeros_like(b)
    st, info = binding.qcd_solve(lat.ctx, b, x, 1, binding.solver_params(tol=1e-10, nkv=2, max_restarts=2),
                                 raise_on_fail=False)
    assert st == -8 and info[0]["restarts"] == 2  # QCD_NOT_CONVERGED
    A = orc.clover(dims, U, 0.0, 1.5)
    res = np.linalg.norm(bn - orc.apply_D(dims, U, A, AP, x.cpu().numpy())) / np.linalg.norm(bn)
    assert 1e-10 < res < 1.0 and abs(res - info[0]["true_residual"]) < 1e-10
    lat.close()


def test_ragged_lattice_and_blocks(orc):
    """Every extent and block extent different (8 x 12 x 4 x 16 with 4 x 6 x 2 x 4
    blocks): solve to 1e-10 against the oracle's operator."""
    dims, block = (8, 12, 4, 16), (4, 6, 2, 4)
    lat, U, rng = _lat(dims, block, m0=-0.1)
    bn = synth.gaussian_spinor(dims, rng)
    x, info = lat.solve(torch.from_numpy(bn).cuda(), tol=1e-10, sap_prec="f16")
    assert info[0]["status"] == 0
    A = orc.clover(dims, U, -0.1, 1.5)
    res = np.linalg.norm(bn - orc.apply_D(dims, U, A, AP, x.cpu().numpy())) / np.linalg.norm(bn)
    assert res <= 1.05e-10
    lat.close()


def test_solves_are_deterministic():
    """Fixed grids, fixed-order reductions and face buffers instead of atomics:
    repeating a solve reproduces it bit for bit."""
    dims = (16, 8, 8, 16)
    lat, U, rng = _lat(dims, (4, 4, 4, 4))
    b = torch.from_numpy(synth.gaussian_spinor(dims, rng)).cuda()
    x1, i1 = lat.solve(b, tol=1e-10, sap_prec="f16")
    x2, i2 = lat.solve(b, tol=1e-10, sap_prec="f16")
    assert torch.equal(x1, x2) and i1[0]["iterations"] == i2[0]["iterations"]
    lat.close()


def test_zero_guess_ignores_the_input_x():
    """zero_guess = 1 starts from x = 0 whatever x holds (here NaN), for device
    and host buffers and for the adjoint solve: the same iterates, bit for bit,
    as a solve whose x holds zeros."""
    from paper_1109_4279_gb300 import binding
    dims = (8, 8, 8, 8)
    lat, U, rng = _lat(dims, (4, 4, 2, 2))
    bn = synth.gaussian_spinor(dims, rng)
    nan = complex(float("nan"), float("nan"))
    sp0 = binding.solver_params(tol=1e-10, sap_prec="f16")
    sp1 = binding.solver_params(tol=1e-10, sap_prec="f16", zero_guess=1)
    b = torch.from_numpy(bn).cuda()
    x_ref = torch.zeros_like(b)
    _, i_ref = binding.qcd_solve(lat.ctx, b, x_ref, 1, sp0)
    for dev in (True, False):
        bb = b if dev else b.cpu()
        x = torch.full_like(bb, nan)
        st, info = binding.qcd_solve(lat.ctx, bb, x, 1, sp1, raise_on_fail=False)
        assert st == 0 and info[0]["iterations"] == i_ref[0]["iterations"]
        assert torch.equal(x.cpu(), x_ref.cpu())
    y_ref = torch.zeros_like(b)
    binding.qcd_solve_dagger(lat.ctx, b, y_ref, sp0)
    y = torch.full_like(b, nan)
    st, _ = binding.qcd_solve_dagger(lat.ctx, b, y, sp1, raise_on_fail=False)
    assert st == 0 and torch.equal(y, y_ref)
    lat.close()


def test_zero_guess_with_several_right_hand_sides_on_host(orc):
    """nrhs = 2 from host buffers with zero_guess: both converge against the
    oracle's operator although x holds NaN."""
    from paper_1109_4279_gb300 import binding
    dims = (8, 8, 8, 8)
    lat, U, rng = _lat(dims, (4, 4, 2, 2))
    bn = synth.gaussian_spinor(dims, rng, nrhs=2)
    b = torch.from_numpy(bn)
    x = torch.full_like(b, complex(float("nan"), float("nan")))
    st, info = binding.qcd_solve(lat.ctx, b, x, 2, binding.solver_params(tol=1e-10, sap_prec="f16", zero_guess=1),
                                 raise_on_fail=False)
    assert st == 0 and [i["status"] for i in info] == [0, 0]
    A = orc.clover(dims, U, 0.0, 1.5)
    for k in range(2):
        r = bn[k] - orc.apply_D(dims, U, A, AP, x[k].numpy())
        assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(bn[k])
    lat.close()


@pytest.mark.parametrize("dims,block,nkv", [((16, 8, 8, 8), (4, 4, 4, 4), 16), ((12, 8, 8, 8), (2, 4, 4, 4), 16),
                                            ((16, 8, 8, 8), (4, 4, 4, 4), 2)])
def test_host_buffers_match_device_buffers(orc, dims, block, nkv):
    """A single right-hand side from host memory (pinned, with and without an
    initial guess) goes up and comes back in slabs of time slices, copies
    overlapped with the layout kernels, and every restart's x is handed to the
    caller while the residual is computed: the solution equals the one from
    device buffers bit for bit and meets the oracle's residual (16 / 4 = 4
    slabs; 12 / 2 = 6 slabs; nkv = 2: many restarts, each delivering x)."""
    from paper_1109_4279_gb300 import binding
    lat, U, rng = _lat(dims, block)
    bn = synth.gaussian_spinor(dims, rng)
    x0n = 0.1 * synth.gaussian_spinor(dims, rng)
    A = orc.clover(dims, U, 0.0, 1.5)
    for guess in (False, True):
        kw = dict(tol=1e-10, nkv=nkv, sap_prec="f16", outer_prec="df64", zero_guess=0 if guess else 1)
        bd = torch.from_numpy(bn).cuda()
        xd = torch.from_numpy(x0n).cuda() if guess else torch.zeros_like(bd)
        st, _ = binding.qcd_solve(lat.ctx, bd, xd, 1, binding.solver_params(**kw))
        bh = torch.from_numpy(bn).pin_memory()
        xh = torch.from_numpy(x0n).pin_memory() if guess else torch.full_like(bh, float("nan")).pin_memory()
        st, info = binding.qcd_solve(lat.ctx, bh, xh, 1, binding.solver_params(**kw))
        assert np.array_equal(xh.numpy(), xd.cpu().numpy()), guess
        res = np.linalg.norm(bn - orc.apply_D(dims, U, A, AP, xh.numpy())) / np.linalg.norm(bn)
        assert res <= 1.05e-10 and abs(res - info[0]["true_residual"]) < 1e-13, (guess, info)
        if nkv == 2:
            assert info[0]["restarts"] > 2
    lat.close()


def test_sap_staging_wait_runs_out_and_the_context_recovers(orc):
    """A staging barrier told to expect 16 bytes more than its copies deliver
    never completes: every block's bounded wait runs out (the drain wait after
    it takes about a second), the kernel records it and returns, and
    qcd_sap_apply and qcd_solve report QCD_ERR_TIMEOUT.  With the hook
    cleared, the same context reproduces the oracle's SAP and solves."""
    import ctypes
    from paper_1109_4279_gb300 import binding
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    lat, U, rng = _lat(dims, block)
    bn = synth.gaussian_spinor(dims, rng)
    b = torch.from_numpy(bn).cuda()
    psi = torch.empty_like(b)
    binding.qcd_debug_set(lat.ctx, "sap_extra_tx", 16)
    binding.qcd_debug_set(lat.ctx, "sap_wait_cycles", 1 << 20)
    st = binding.lib().qcd_sap_apply(lat.ctx, binding._ptr(b), binding._ptr(psi), 1, 4, 2, binding._stream())
    assert st == -13  # QCD_ERR_TIMEOUT
    x = torch.zeros_like(b)
    st, info = binding.qcd_solve(lat.ctx, b, x, 1, binding.solver_params(tol=1e-10, sap_prec="f16", ncy=1, nkv=1,
                                                                         max_restarts=1), raise_on_fail=False)
    assert st == -13 and info[0]["status"] == -13
    for what, value in (("sap_extra_tx", -1), ("sap_wait_cycles", 0), (7, 1)):
        assert binding.lib().qcd_debug_set(lat.ctx, binding.DEBUG.get(what, what), ctypes.c_longlong(value)) == -1
    binding.qcd_debug_set(lat.ctx, "sap_extra_tx", 0)
    binding.qcd_debug_set(lat.ctx, "sap_wait_cycles", 1 << 31)
    out = lat.sap(b, ncy=4, nmr=4, prec="f16").cpu().numpy()
    A = orc.clover(dims, U, 0.0, 1.5)
    assert rel(out, orc.sap(dims, U, A, AP, block, bn, ncy=4, nmr=4)) < 5e-3
    x, info = lat.solve(b, tol=1e-10, sap_prec="f16")
    assert info[0]["status"] == 0
    assert np.linalg.norm(bn - orc.apply_D(dims, U, A, AP, x.cpu().numpy())) <= 1.05e-10 * np.linalg.norm(bn)
    lat.close()
