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


@pytest.mark.parametrize("prec,dims,block", [("f16", (16, 8, 8, 8), (8, 4, 4, 4)), ("f32", (8, 8, 8, 16), (4, 4, 4, 4)),
                                             ("f64", (8, 8, 8, 8), (4, 4, 2, 2))])
def test_tiled_sap_matches_oracle(orc, prec, dims, block):
    """The RHS-tiled SAP kernel (a CTA stages its block's links and clover once
    and solves a tile of right-hand sides in turn): five right-hand sides with
    tiles of 1, 2 and 5 give, for every right-hand side, the oracle's M_SAP at
    the block-field tolerance; the tile size does not change a single bit, and
    the untiled single-right-hand-side kernel agrees."""
    from paper_1109_4279_gb300 import binding as B
    U, rng = synth.gauge_field(dims, 0.5, 95)
    eta = synth.gaussian_spinor(dims, rng, nrhs=5)
    m0, csw = -0.05, 1.5
    lat = B.Lattice(dims, block, m0, csw)
    lat.load_gauge(torch.from_numpy(U).cuda())
    A = orc.clover(dims, U, m0, csw)
    et = torch.from_numpy(eta).cuda()
    outs = {}
    for rt in (1, 2, 5):
        psi = torch.empty_like(et)
        B.qcd_sap_apply_n(lat.ctx, et, psi, 5, rt, 4, 4, prec)
        outs[rt] = psi.cpu().numpy()
    assert np.array_equal(outs[1], outs[2]) and np.array_equal(outs[1], outs[5])
    tol = {"f64": 1e-12, "f32": 1e-5, "f16": 5e-3}[prec]
    for q in range(5):
        ref = orc.sap(dims, U, A, AP, block, eta[q], ncy=4, nmr=4)
        assert rel(outs[2][q], ref) < tol, q
        single = lat.sap(et[q].contiguous(), ncy=4, nmr=4, prec=prec).cpu().numpy()
        assert rel(outs[2][q], single) < {"f64": 1e-14, "f32": 1e-6, "f16": 1e-6}[prec], q
    lat.close()


@pytest.mark.parametrize("outer_prec", ["f64", "df64"])
def test_tiled_solve_with_uneven_convergence(orc, outer_prec):
    """Three right-hand sides iterated by the same launches whose cycles end at
    different iterations: a Gaussian source from x = 0, a point source from a
    rough solution (1e-4), and b = 0, which is solved by x = 0 without
    iterating; the device mask switches off each one as its cycle ends.  Every
    solution against the oracle's operator and against the same right-hand
    side solved alone from the same initial guess."""
    from paper_1109_4279_gb300 import binding as B
    dims, block, m0, csw = (8, 8, 8, 8), (4, 4, 2, 2), -0.1, 1.5
    U, rng = synth.gauge_field(dims, 0.5, 96)
    b = np.zeros((3,) + (synth.volume(dims), 4, 3), np.complex128)
    b[0] = synth.gaussian_spinor(dims, rng)
    b[1] = synth.point_sources(dims, site=77)[5]
    lat = B.Lattice(dims, block, m0, csw)
    lat.load_gauge(torch.from_numpy(U).cuda())
    bt = torch.from_numpy(b).cuda()
    x0 = torch.zeros_like(bt)
    x0[1], _ = lat.solve(bt[1].contiguous(), tol=1e-4, sap_prec="f16")
    x, info = lat.solve(bt, x0=x0, tol=1e-10, sap_prec="f16", nkv=16, outer_prec=outer_prec)
    assert all(i["status"] == 0 for i in info), info
    assert info[2]["iterations"] == 0 and info[1]["iterations"] < info[0]["iterations"], info
    x = x.cpu().numpy()
    assert not np.any(x[2])
    A = orc.clover(dims, U, m0, csw)
    for q in range(2):
        assert _res(orc, dims, U, A, b[q], x[q]) <= 1.05e-10
        xs, inf1 = lat.solve(bt[q].contiguous(), x0=x0[q].contiguous(), tol=1e-10, sap_prec="f16", nkv=16,
                             outer_prec=outer_prec)
        assert abs(inf1[0]["iterations"] - info[q]["iterations"]) <= 1
        assert rel(x[q], xs.cpu().numpy()) < 1e-8
    lat.close()
