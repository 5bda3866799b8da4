"""GPU autotuning: the operator's launch shape per precision (CTA size, and
one or two threads per site for 16-bit storage), the batched SAP sweep's
right-hand-side tile (cached in a JSON file), and the Schwarz block shape
chosen by timing complete solves."""
import json

import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T


def test_autotune_cache_and_parity(orc, tmp_path):
    from paper_1109_4279_gb300 import binding as B
    dims, block = (32, 16, 16, 16), (4, 4, 4, 4)
    U, rng = synth.gauge_field(dims, 0.5, 2)
    b = synth.gaussian_spinor(dims, rng)
    lat = B.Lattice(dims, block, 0.0, 1.5)
    lat.load_gauge(torch.from_numpy(U).cuda())
    cache = str(tmp_path / "tune.json")
    B.qcd_autotune(lat.ctx, 1, cache)
    entries = json.load(open(cache))
    assert len(entries) == 1
    (key, vals), = entries.items()
    # CTA sizes of the five precisions (double-float last), threads per site
    # of the two 16-bit operators, SAP right-hand-side tile (0: default)
    assert "16x16" in key and len(vals) == 8
    assert all(v in (128, 256, 512) for v in vals[:4]) and vals[4] in (128, 256)
    assert vals[5] in (1, 2) and vals[6] in (1, 2) and vals[7] == 0
    assert B.qcd_get_launch(lat.ctx, "f16")[:2] == (vals[2] if vals[5] == 1 else 256, vals[5])
    B.qcd_autotune(lat.ctx, 1, cache)  # second call applies the cached entry
    assert json.load(open(cache)) == entries
    A = orc.clover(dims, U, 0.0, 1.5)
    ref = orc.apply_D(dims, U, A, AP, b)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5), ("f16", 5e-3), ("df64", 1e-12)):
        out = lat.apply_D(torch.from_numpy(b).cuda(), prec=prec).cpu().numpy()
        assert rel(out, ref) < tol
    lat.close()


def test_tune_block_shape():
    """4^4 versus 8x4x4x4 blocks on the 16^3 x 32 lattice: both solve, the
    fastest is returned."""
    from paper_1109_4279_gb300 import binding as B
    dims = (32, 16, 16, 16)
    U, rng = synth.gauge_field(dims, 0.5, 2)
    b = synth.gaussian_spinor(dims, rng)
    cands = [(4, 4, 4, 4), (8, 4, 4, 4)]
    best, times = B.qcd_tune_block(dims, 0.0, 1.5, torch.from_numpy(U).cuda(), torch.from_numpy(b).cuda(), cands,
                                   B.solver_params(tol=1e-10, sap_prec="f16"))
    assert best in cands
    assert all(t > 0 for t in times.values()), times
    assert times[best] == min(times.values())


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("dims,block", [((16, 8, 8, 8), (8, 4, 4, 4)), ((8, 8, 8, 16), (4, 4, 4, 4)),
                                        ((8, 12, 4, 8), (4, 6, 2, 2))])
def test_two_threads_per_site_operator(orc, prec, dims, block):
    """The 16-bit operator with two threads per site (each thread two of the
    four directions and half of the spin components), D and D^+, three
    right-hand sides in one launch, against the oracle at the 16-bit
    tolerance, and against the one-thread form."""
    from paper_1109_4279_gb300 import binding as B
    U, rng = synth.gauge_field(dims, 0.5, 97)
    b = synth.gaussian_spinor(dims, rng, nrhs=3)
    lat = B.Lattice(dims, block, -0.05, 1.5)
    lat.load_gauge(torch.from_numpy(U).cuda())
    A = orc.clover(dims, U, -0.05, 1.5)
    bt = torch.from_numpy(b).cuda()
    for dagger in (False, True):
        B.qcd_set_launch(lat.ctx, prec, 256, 2)
        assert B.qcd_get_launch(lat.ctx, prec) == (256, 2)
        two = lat.apply_D(bt, dagger=dagger, prec=prec).cpu().numpy()
        B.qcd_set_launch(lat.ctx, prec, 256, 1)
        one = lat.apply_D(bt, dagger=dagger, prec=prec).cpu().numpy()
        for q in range(3):
            ref = orc.apply_D(dims, U, A, AP, b[q], dagger=dagger)
            assert rel(two[q], ref) < 5e-3
            assert rel(two[q], one[q]) < 1e-3
    assert B.lib().qcd_set_launch(lat.ctx, B.PREC["f32"], 256, 2) == -11  # QCD_ERR_UNSUPPORTED
    lat.close()


def test_autotune_sap_tile_for_many_rhs(tmp_path):
    """With 12 right-hand sides the autotuner also times the batched SAP
    sweep's right-hand-side tile; the tile is kept, cached, and can be pinned."""
    from paper_1109_4279_gb300 import binding as B
    dims, block = (16, 8, 8, 8), (8, 4, 4, 4)
    U, _ = synth.gauge_field(dims, 0.5, 98)
    lat = B.Lattice(dims, block, 0.0, 1.5)
    lat.load_gauge(torch.from_numpy(U).cuda())
    cache = str(tmp_path / "tune12.json")
    B.qcd_autotune(lat.ctx, 12, cache)
    (key, vals), = json.load(open(cache)).items()
    assert "nrhs12" in key and vals[7] in (1, 2, 3, 4, 6, 8, 12)
    assert B.qcd_get_sap_tile(lat.ctx, 12) == vals[7]
    B.qcd_set_sap_tile(lat.ctx, 5)
    assert B.qcd_get_sap_tile(lat.ctx, 12) == 5 and B.qcd_get_sap_tile(lat.ctx, 3) == 3
    B.qcd_set_sap_tile(lat.ctx, 0)
    assert B.qcd_get_sap_tile(lat.ctx, 1) == 1
    lat.close()
