"""GPU autotuning: the operator's CTA size per precision (cached in a JSON
file) and the Schwarz block shape chosen by timing complete solves."""
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
    assert "16x16" in key and all(v in (128, 256, 512) for v in vals)
    B.qcd_autotune(lat.ctx, 1, cache)  # second call applies the cached entry
    assert json.load(open(cache)) == entries
    A = orc.clover(dims, U, 0.0, 1.5)
    ref = orc.apply_D(dims, U, A, AP, b)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5), ("f16", 5e-3)):
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
