"""The precision codecs between the FP64 recursion and the FP32 preconditioner
(Sec. 4) convert with integer operations; they must give exactly the hardware
conversions: FP64 -> FP32 rounded to nearest even (including halfway cases,
overflow to infinity, subnormal results, signed zeros, infinities and NaN) and
the exact FP32 -> FP64 widening (including subnormal inputs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _f64_cases(rng):
    bits = rng.integers(0, 2 ** 63, size=200000, dtype=np.int64).astype(np.uint64)
    bits |= rng.integers(0, 2, size=bits.size, dtype=np.uint64) << np.uint64(63)
    rand = bits.view(np.float64)
    # values near every FP32 rounding boundary: FP32 numbers x, x +- half an
    # ulp exactly (ties), and one FP64 ulp either side of the tie
    f = rng.standard_normal(20000).astype(np.float32) * np.float32(2.0) ** rng.integers(-60, 60, 20000).astype(np.float32)
    f = f.astype(np.float64)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    tie = np.concatenate([f + ulp / 2, f - ulp / 2])
    near = np.concatenate([np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf), tie, f])
    fmax = float(np.finfo(np.float32).max)
    fmin = float(np.finfo(np.float32).tiny)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax * (1 + 2 ** -25), fmax * (1 + 2 ** -24),
                        2.0 ** 128, fmin, fmin * (1 - 2 ** -25), fmin / 2, fmin * 2 ** -23, fmin * 2 ** -24,
                        fmin * 2 ** -25, 5e-324, 1e-310, 1.0, -1.0, 1 + 2 ** -24, 1 + 3 * 2 ** -24, 1e300, -1e-300])
    return np.concatenate([rand, near, special])


def _f32_cases(rng):
    bits = rng.integers(0, 2 ** 32, size=200000, dtype=np.int64).astype(np.uint32)
    special = np.array([0, 0x80000000, 1, 0x807fffff, 0x00800000, 0x7f7fffff, 0x7f800000, 0xff800000, 0x7fc00000,
                        0x3f800000], dtype=np.uint32)
    return np.concatenate([bits, special]).view(np.float32)


def test_conversions_match_hardware():
    from paper_1109_4279_gb300 import binding
    rng = np.random.default_rng(1234)
    a64 = _f64_cases(rng)
    a32 = _f32_cases(rng)
    n = min(a64.size, a32.size)
    in64 = torch.from_numpy(a64[:n].copy()).cuda()
    in32 = torch.from_numpy(a32[:n].copy()).cuda()
    tail64 = torch.from_numpy(a64[n:].copy()).cuda()
    out32 = torch.empty(n, dtype=torch.float32, device="cuda")
    out64 = torch.empty(n, dtype=torch.float64, device="cuda")
    binding.qcd_convert_check(in64, in32, out32, out64)
    ref32 = in64.to(torch.float32)
    ref64 = in32.to(torch.float64)
    torch.cuda.synchronize()
    for got, ref in ((out32, ref32), (out64, ref64)):
        nan = torch.isnan(ref)
        assert torch.equal(torch.isnan(got), nan)
        itype = torch.int32 if got.dtype == torch.float32 else torch.int64
        assert torch.equal(got[~nan].view(itype), ref[~nan].view(itype))
    # the rest of the FP64 cases (more of them than FP32 ones)
    m = tail64.numel()
    o32 = torch.empty(m, dtype=torch.float32, device="cuda")
    o64 = torch.empty(m, dtype=torch.float64, device="cuda")
    binding.qcd_convert_check(tail64, torch.zeros(m, dtype=torch.float32, device="cuda"), o32, o64)
    r32 = tail64.to(torch.float32)
    torch.cuda.synchronize()
    nan = torch.isnan(r32)
    assert torch.equal(torch.isnan(o32), nan)
    assert torch.equal(o32[~nan].view(torch.int32), r32[~nan].view(torch.int32))


def test_convert_check_arguments():
    from paper_1109_4279_gb300 import binding
    st = binding.lib().qcd_convert_check(None, None, None, None, -1, None)
    assert st == -1
    assert binding.lib().qcd_convert_check(None, None, None, None, 0, None) == 0
