"""The allocation-free operator apply (qcd_apply_D_noalloc) through the C ABI.

Some callers cannot let a library allocate device memory: programs whose own
pool allocator owns all of it, and latency-bound loops in which cudaFree's
device-wide synchronisation would stall other streams.  For them the FP64
apply keeps its two staging fields in a static device array of the library
(at most 65536 sites).  This file is collected last so that a failure here,
under -x, comes after every other test has run.
"""
import numpy as np
import pytest

from helpers import rel
from paper_1109_4279_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AP = synth.ANTIPERIODIC_T


def test_no_alloc_apply_matches_apply_D_and_oracle_twice(orc):
    """Two calls in a row (different inputs, D then D^+) equal qcd_apply_D and
    the oracle's D / D^+ at the FP64 parity tolerance; the second call reuses
    the shared array."""
    from paper_1109_4279_gb300 import binding as B
    dims, block, m0, csw = (8, 8, 8, 16), (4, 4, 4, 4), 0.0, 1.5
    U, rng = synth.gauge_field(dims, 0.5, 81)
    lat = B.Lattice(dims, block, m0, csw)
    lat.load_gauge(torch.from_numpy(U).cuda())
    A = orc.clover(dims, U, m0, csw)
    for dagger in (False, True):
        bn = synth.gaussian_spinor(dims, rng)
        b = torch.from_numpy(bn).cuda()
        out = torch.empty_like(b)
        st = B.qcd_apply_D_noalloc(lat.ctx, b, out, dagger)
        assert st == 0, B.qcd_status_string(st)
        ref = torch.empty_like(b)
        B.qcd_apply_D(lat.ctx, b, ref, dagger, "f64", 1)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert rel(o, ref.cpu().numpy()) < 1e-12
        assert rel(o, orc.apply_D(dims, U, A, AP, bn, dagger=dagger)) < 1e-12
    lat.close()


def test_no_alloc_leaves_free_memory_unchanged():
    """After the first call (which may load the library's device module and
    look up the array's address), further calls change the device's free
    memory by nothing: every buffer they touch already exists."""
    from paper_1109_4279_gb300 import binding as B
    dims, block = (16, 8, 8, 8), (4, 4, 4, 4)
    U, rng = synth.gauge_field(dims, 0.5, 82)
    lat = B.Lattice(dims, block, 0.1, 1.0)
    lat.load_gauge(torch.from_numpy(U).cuda())
    b = torch.from_numpy(synth.gaussian_spinor(dims, rng)).cuda()
    out1, out2 = torch.empty_like(b), torch.empty_like(b)
    assert B.qcd_apply_D_noalloc(lat.ctx, b, out1, False) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(3):
        assert B.qcd_apply_D_noalloc(lat.ctx, b, out2, k % 2 == 1) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert B.qcd_apply_D_noalloc(lat.ctx, b, out2, False) == 0
    torch.cuda.synchronize()
    assert torch.equal(out1, out2)
    lat.close()


def test_no_alloc_rejects_too_large_and_profiling():
    from paper_1109_4279_gb300 import binding as B
    lat = B.Lattice((32, 16, 16, 16), (4, 4, 4, 4), 0.0, 1.5)  # 131072 sites > 65536
    x = torch.zeros((lat.V, 4, 3), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    assert B.qcd_apply_D_noalloc(lat.ctx, x, y, False) == -12  # QCD_ERR_TOO_LARGE
    lat.close()
    dims = (8, 8, 8, 8)
    U, _ = synth.gauge_field(dims, 0.5, 83)
    lat = B.Lattice(dims, (4, 4, 2, 2), 0.0, 1.5)
    lat.load_gauge(torch.from_numpy(U).cuda())
    x = torch.zeros((lat.V, 4, 3), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    B.qcd_profile_enable(lat.ctx, True)
    assert B.qcd_apply_D_noalloc(lat.ctx, x, y, False) == -5  # QCD_ERR_STATE: profiling creates events
    B.qcd_profile_enable(lat.ctx, False)
    assert B.qcd_apply_D_noalloc(lat.ctx, x, y, False) == 0
    lat.close()
