"""Parity at the full size of the benchmarked workload: the 32^3 x 64 lattice
(links exp(i 0.5 sum_a g_a lambda_a / 2) from seed 3, m0 = -0.05, c_sw = 1.5,
antiperiodic time) with 8 x 4 x 4 x 4 Schwarz blocks, in the configuration the
benchmark times.  The oracle finishes the whole-field operator and one SAP
application in seconds here, so these compare every element; the solve is
checked through its defining property, the true residual recomputed with the
oracle's operator, and element by element against the oracle's own solution
(about two minutes of oracle GCR on the host cores).
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T
DIMS, BLOCK, M0, CSW = (64, 32, 32, 32), (8, 4, 4, 4), -0.05, 1.5


@pytest.fixture(scope="module")
def full(orc):
    from paper_1109_4279_gb300 import binding
    U, rng = synth.gauge_field(DIMS, 0.5, 3)
    b = synth.gaussian_spinor(DIMS, rng)
    lat = binding.Lattice(DIMS, BLOCK, M0, CSW)
    lat.load_gauge(torch.from_numpy(U).cuda())
    A = orc.clover(DIMS, U, M0, CSW)
    yield U, A, b, lat
    lat.close()


def test_full_size_operator(orc, full):
    U, A, b, lat = full
    ref = orc.apply_D(DIMS, U, A, AP, b)
    bt = torch.from_numpy(b).cuda()
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5), ("f16", 5e-3)):
        out = lat.apply_D(bt, prec=prec).cpu().numpy()
        assert rel(out, ref) < tol, prec


def test_full_size_sap(orc, full):
    U, A, b, lat = full
    psi = lat.sap(torch.from_numpy(b).cuda(), ncy=4, nmr=4, prec="f16").cpu().numpy()
    ref = orc.sap(DIMS, U, A, AP, BLOCK, b, ncy=4, nmr=4)
    assert rel(psi, ref) < 5e-3


@pytest.fixture(scope="module")
def full_solution(orc, full):
    """The oracle's solution: unpreconditioned FP64 GCR(16) to 1e-12."""
    U, A, b, lat = full
    x_or, _, _, conv, res_or = orc.fgcr(DIMS, U, A, AP, b, nkv=16, tol=1e-12, max_restarts=400)
    assert conv and res_or <= 1e-12
    return x_or


@pytest.mark.parametrize("outer_prec", ["f64", "df64"])
def test_full_size_solve(orc, full, full_solution, outer_prec):
    """The benchmarked solve (FP16 block fields, tolerance 1e-10) with the FP64
    and the double-float recursion: its true residual, recomputed with the
    oracle's operator, and its solution against the oracle's."""
    U, A, b, lat = full
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, sap_prec="f16", outer_prec=outer_prec)
    assert info[0]["status"] == 0
    x = x.cpu().numpy()
    res = np.linalg.norm(b - orc.apply_D(DIMS, U, A, AP, x)) / np.linalg.norm(b)
    assert res <= 1.05e-10
    assert abs(res - info[0]["true_residual"]) < 1e-12
    assert rel(x, full_solution) < 1e-8
