"""GPU batched solves: many right-hand sides on one lattice and one right-hand
side on each of several lattices of different sizes, solved in lock step
(concurrent streams, CUDA-graph replay of each iteration).  Every solution is
checked with the oracle's operator: |b - D x| / |b| <= 1e-10 per problem, and
the batched result equals the one-at-a-time solve.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T


def _res(orc, dims, U, A, b, x):
    return np.linalg.norm(b - orc.apply_D(dims, U, A, AP, x)) / np.linalg.norm(b)


def test_twelve_point_sources(orc):
    """12 spin-colour point sources at site 0 (the multi-RHS workload's sources)
    on an 8^3 x 16 lattice, nrhs = 12 in one call."""
    from paper_1109_4279_gb300 import binding as B
    dims, block = (16, 8, 8, 8), (4, 4, 4, 4)
    U, _ = synth.gauge_field(dims, 0.5, 4)
    b = synth.point_sources(dims)
    lat = B.Lattice(dims, block, 0.0, 1.5)
    lat.load_gauge(torch.from_numpy(U).cuda())
    bt = torch.from_numpy(b).cuda()
    x, info = lat.solve(bt, tol=1e-10, sap_prec="f16")
    assert len(info) == 12 and all(i["status"] == 0 for i in info), info
    x = x.cpu().numpy()
    A = orc.clover(dims, U, 0.0, 1.5)
    for k in range(12):
        assert _res(orc, dims, U, A, b[k], x[k]) <= 1.05e-10
    # one right-hand side alone gives the same solution
    x3, _ = lat.solve(bt[3].contiguous(), tol=1e-10, sap_prec="f16")
    assert np.linalg.norm(x3.cpu().numpy() - x[3]) <= 1e-12 * np.linalg.norm(x[3])
    lat.close()


def test_uneven_lattices_batch(orc):
    """Ten lattices of four sizes (2 x 8^4, 2 x 8^3x16, 3 x 12^3x24, 3 x 16^3x32;
    seeds 10..19) in one qcd_solve_batch call, each with its own block shape."""
    from paper_1109_4279_gb300 import binding as B
    blocks = {(8, 8, 8, 8): (4, 4, 2, 2), (16, 8, 8, 8): (4, 4, 4, 4), (24, 12, 12, 12): (4, 6, 2, 2),
              (32, 16, 16, 16): (4, 4, 4, 4)}
    lats, bs, xs, fields = [], [], [], []
    for k, dims in enumerate(synth.UNEVEN_LATTICES):
        U, rng = synth.gauge_field(dims, 0.5, 10 + k)
        b = synth.gaussian_spinor(dims, rng)
        lat = B.Lattice(dims, blocks[dims], 0.0, 1.5)
        lat.load_gauge(torch.from_numpy(U).cuda())
        lats.append(lat)
        bs.append(torch.from_numpy(b).cuda())
        xs.append(torch.zeros_like(bs[-1]))
        fields.append((dims, U, b))
    st, info = B.qcd_solve_batch([l.ctx for l in lats], bs, xs, B.solver_params(tol=1e-10, sap_prec="f16"))
    assert st == 0 and all(i["status"] == 0 for i in info), info
    for (dims, U, b), x in zip(fields, xs):
        A = orc.clover(dims, U, 0.0, 1.5)
        assert _res(orc, dims, U, A, b, x.cpu().numpy()) <= 1.05e-10
    for lat in lats:
        lat.close()


def test_batched_solve_after_new_gauge_field(orc):
    """Batched solves replay captured per-iteration graphs.  Loading a second
    gauge field and rebuilding the clover term reallocates the operator data
    those graphs were captured with; the next batched solve with the same
    parameters must run on the new field (true residual of the new operator,
    recomputed by the oracle)."""
    from paper_1109_4279_gb300 import binding as B
    dims, block, m0, csw = (8, 8, 8, 8), (4, 4, 2, 2), 0.0, 1.5
    lat = B.Lattice(dims, block, m0, csw)
    rng = np.random.default_rng(91)
    b = synth.gaussian_spinor(dims, rng, nrhs=2)
    bt = torch.from_numpy(b).cuda()
    for seed in (92, 93):
        U, _ = synth.gauge_field(dims, 0.5, seed)
        lat.load_gauge(torch.from_numpy(U).cuda())
        x, info = lat.solve(bt, tol=1e-10, sap_prec="f16")
        assert all(i["status"] == 0 for i in info), info
        A = orc.clover(dims, U, m0, csw)
        x = x.cpu().numpy()
        for k in range(2):
            assert _res(orc, dims, U, A, b[k], x[k]) <= 1.05e-10
    lat.close()


def test_twelve_point_sources_full_24x48(orc):
    """The multi-right-hand-side workload at full size: the 12 spin-colour
    point sources on 24^3 x 48 (seed 4, eps 0.5, m0 0, c_sw 1.5; FP16 block
    fields, FP64 recursion) in one call.  Every solution's true residual is
    recomputed with the oracle's operator, and the first source's solution
    (a column of the propagator) is compared with the oracle's GCR solution."""
    from paper_1109_4279_gb300 import binding as B
    w = synth.WORKLOADS["24^3x48 12 point sources"]
    dims = w["dims"]
    U, _ = synth.gauge_field(dims, w["eps"], w["seed"])
    b = synth.point_sources(dims)
    lat = B.Lattice(dims, w["block"], w["m0"], w["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    x, info = lat.solve(torch.from_numpy(b).cuda(), tol=1e-10, nkv=w["nkv"], ncy=w["ncy"], nmr=w["nmr"],
                        sap_prec="f16")
    assert len(info) == 12 and all(i["status"] == 0 for i in info), info
    x = x.cpu().numpy()
    lat.close()
    A = orc.clover(dims, U, w["m0"], w["csw"])
    for k in range(12):
        assert _res(orc, dims, U, A, b[k], x[k]) <= 1.05e-10, k
    x_or, _, _, conv, res_or = orc.fgcr(dims, U, A, AP, b[0], nkv=16, tol=1e-12, max_restarts=400)
    assert conv and res_or <= 1e-12
    assert rel(x[0], x_or) < 1e-8
