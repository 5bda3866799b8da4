"""ctypes binding of libqcdgb (include/qcdgb.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; tensors
are torch tensors on the GPU (complex128 spinors/links, float64 forces) whose
device pointers and the current CUDA stream are passed through.  There is no
fallback: if libqcdgb.so is missing this module raises on first use.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqcdgb.so")

QCD_OK = 0
STATUS = {
    0: "QCD_OK", -1: "QCD_ERR_ARG", -2: "QCD_ERR_GEOMETRY", -3: "QCD_ERR_CUDA", -4: "QCD_ERR_NOMEM",
    -5: "QCD_ERR_STATE", -6: "QCD_ERR_NOT_SU3", -7: "QCD_ERR_SINGULAR_CLOVER", -8: "QCD_NOT_CONVERGED",
    -9: "QCD_STAGNATED", -10: "QCD_NAN", -11: "QCD_ERR_UNSUPPORTED", -12: "QCD_ERR_TOO_LARGE",
    -13: "QCD_ERR_TIMEOUT",
}
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "df64": 4}
PRECOND = {"none": 0, "sap": 1}
SOLVER = {"fgcr": 0, "fgmres_dr": 1, "cg": 2, "cg_eo": 3}
KERNEL = {"dirac": 0, "sap": 1, "blas": 2, "residual": 3}


class QcdError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = "%s failed: %s (%s)" % (what, STATUS.get(status, status), _status_string(status))
        if status == -3:
            msg += ": " + lib().qcd_last_error().decode()
        super().__init__(msg)


class Params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("block", ctypes.c_int * 4), ("m0", ctypes.c_double),
                ("csw", ctypes.c_double), ("bc", ctypes.c_double * 4)]


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("nkv", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("precond", ctypes.c_int), ("ncy", ctypes.c_int), ("nmr", ctypes.c_int),
                ("sap_prec", ctypes.c_int), ("outer_prec", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("solver", ctypes.c_int), ("ndefl", ctypes.c_int), ("cg_fallback", ctypes.c_int),
                ("cg_max_iter", ctypes.c_int), ("zero_guess", ctypes.c_int), ("residual_prec", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("time_ms", ctypes.c_double), ("sap_ms", ctypes.c_double),
                ("dirac_ms", ctypes.c_double), ("blas_ms", ctypes.c_double), ("cg_iterations", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libqcdgb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqcdgb.so is not built (run __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "qcd_solver_defaults": (None, [ctypes.POINTER(SolverParams)]),
            "qcd_create": (I, [ctypes.POINTER(P), ctypes.POINTER(Params)]),
            "qcd_destroy": (None, [P]),
            "qcd_load_gauge": (I, [P, P, I, P]),
            "qcd_build_clover": (I, [P, P]),
            "qcd_apply_D": (I, [P, P, P, I, I, I, P]),
            "qcd_solve": (I, [P, P, P, I, ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo), P]),
            "qcd_solve_dagger": (I, [P, P, P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo), P]),
            "qcd_solve_batch": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P), ctypes.POINTER(P),
                                    ctypes.POINTER(SolverParams), ctypes.POINTER(SolveInfo), P]),
            "qcd_gradient": (I, [P, P, P, P, P, P, ctypes.POINTER(SolverParams), P]),
            "qcd_force": (I, [P, P, P, P, P]),
            "qcd_autotune": (I, [P, I, ctypes.c_char_p]),
            "qcd_tune_block": (I, [ctypes.POINTER(Params), P, P, I, ctypes.POINTER(SolverParams), P, I,
                                   ctypes.POINTER(ctypes.c_int * 4), ctypes.POINTER(ctypes.c_double)]),
            "qcd_status_string": (ctypes.c_char_p, [I]),
            "qcd_last_error": (ctypes.c_char_p, []),
            "qcd_field_create": (I, [P, I, ctypes.POINTER(P)]),
            "qcd_field_create_n": (I, [P, I, I, ctypes.POINTER(P)]),
            "qcd_field_free": (None, [P]),
            "qcd_field_import": (I, [P, P, P, P]),
            "qcd_field_export": (I, [P, P, P, P]),
            "qcd_apply_D_field": (I, [P, P, P, I, P]),
            "qcd_apply_D_noalloc": (I, [P, P, P, I, P]),
            "qcd_sap_apply": (I, [P, P, P, I, I, I, P]),
            "qcd_sap_apply_n": (I, [P, P, P, I, I, I, I, I, P]),
            "qcd_set_launch": (I, [P, I, I, I]),
            "qcd_measure_alu_peaks": (I, [ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D), P]),
            "qcd_get_launch": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
            "qcd_set_sap_tile": (I, [P, I]),
            "qcd_get_sap_tile": (I, [P, I]),
            "qcd_convert_check": (I, [P, P, P, P, ctypes.c_longlong, P]),
            "qcd_debug_set": (I, [P, I, ctypes.c_longlong]),
            "qcd_profile_enable": (I, [P, I]),
            "qcd_launch_count": (ctypes.c_longlong, []),
            "qcd_profile_reset": (I, [P]),
            "qcd_profile_get": (I, [P, I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D),
                                    ctypes.POINTER(D), ctypes.POINTER(D)]),
            "qcd_gauge_action": (I, [P, P, D, ctypes.POINTER(D), P]),
            "qcd_gauge_force": (I, [P, P, D, P, P]),
            "qcd_update_links": (I, [P, P, P, D, P]),
            "qcd_hmc_trajectory": (I, [P, P, P, P, D, D, I, D, ctypes.POINTER(SolverParams),
                                       ctypes.POINTER(HmcInfo), P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _status_string(st):
    return lib().qcd_status_string(int(st)).decode()


def check(st, what):
    if st != QCD_OK:
        raise QcdError(st, what)
    return st


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def solver_params(**kw) -> SolverParams:
    sp = SolverParams()
    lib().qcd_solver_defaults(ctypes.byref(sp))
    for k, v in kw.items():
        if k in ("sap_prec", "outer_prec", "residual_prec") and isinstance(v, str):
            v = PREC[v]
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        if k == "solver" and isinstance(v, str):
            v = SOLVER[v]
        setattr(sp, k, v)
    return sp


# ---------------------------------------------------------------------------
# one Python function per C entry point (same names)
# ---------------------------------------------------------------------------

def qcd_create(dims, block, m0, csw, bc=(-1.0, 1.0, 1.0, 1.0)):
    p = Params()
    p.dims[:] = [int(d) for d in dims]
    p.block[:] = [int(b) for b in block]
    p.m0, p.csw = float(m0), float(csw)
    p.bc[:] = [float(b) for b in bc]
    h = ctypes.c_void_p()
    check(lib().qcd_create(ctypes.byref(h), ctypes.byref(p)), "qcd_create")
    return h


def qcd_destroy(ctx):
    lib().qcd_destroy(ctx)


def qcd_load_gauge(ctx, U):
    """U: (V, 4, 3, 3) complex128 torch tensor, on the GPU or the CPU."""
    assert U.dtype.is_complex and U.is_contiguous()
    return check(lib().qcd_load_gauge(ctx, _ptr(U), int(U.is_cuda), _stream() if U.is_cuda else None),
                 "qcd_load_gauge")


def qcd_build_clover(ctx):
    return check(lib().qcd_build_clover(ctx, _stream()), "qcd_build_clover")


def qcd_apply_D(ctx, inp, out, dagger=False, prec="f64", nrhs=1):
    assert inp.is_cuda and out.is_cuda and inp.is_contiguous() and out.is_contiguous()
    return check(lib().qcd_apply_D(ctx, _ptr(inp), _ptr(out), int(dagger), PREC[prec], int(nrhs), _stream()),
                 "qcd_apply_D")


def qcd_solve(ctx, b, x, nrhs=1, params: SolverParams | None = None, raise_on_fail=True):
    infos = (SolveInfo * nrhs)()
    st = lib().qcd_solve(ctx, _ptr(b), _ptr(x), int(nrhs), ctypes.byref(params) if params else None, infos,
                         _stream() if b.is_cuda else None)
    if raise_on_fail:
        check(st, "qcd_solve")
    return st, [i.as_dict() for i in infos]


def qcd_solve_dagger(ctx, b, x, params: SolverParams | None = None, raise_on_fail=True):
    info = SolveInfo()
    st = lib().qcd_solve_dagger(ctx, _ptr(b), _ptr(x), ctypes.byref(params) if params else None,
                                ctypes.byref(info), _stream())
    if raise_on_fail:
        check(st, "qcd_solve_dagger")
    return st, info.as_dict()


def qcd_solve_batch(ctxs, bs, xs, params: SolverParams | None = None, raise_on_fail=True):
    n = len(ctxs)
    C = (ctypes.c_void_p * n)(*[c.value for c in ctxs])
    B = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    X = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (SolveInfo * n)()
    st = lib().qcd_solve_batch(C, n, B, X, ctypes.byref(params) if params else None, infos, _stream())
    if raise_on_fail:
        check(st, "qcd_solve_batch")
    return st, [i.as_dict() for i in infos]


def qcd_gradient(ctx, phi, dL_dphi=None, dL_dtheta=None, x_out=None, y_out=None, params=None):
    return check(lib().qcd_gradient(ctx, _ptr(phi), _ptr(dL_dphi), _ptr(dL_dtheta), _ptr(x_out), _ptr(y_out),
                                    ctypes.byref(params) if params else None, _stream()), "qcd_gradient")


def qcd_force(ctx, x, y, F):
    return check(lib().qcd_force(ctx, _ptr(x), _ptr(y), _ptr(F), _stream()), "qcd_force")


def qcd_autotune(ctx, nrhs=1, cache_path=None):
    return check(lib().qcd_autotune(ctx, int(nrhs), cache_path.encode() if cache_path else None), "qcd_autotune")


def qcd_tune_block(dims, m0, csw, U, b, candidates=None, params=None, bc=(-1.0, 1.0, 1.0, 1.0)):
    """Time complete solves over Schwarz block shapes; returns (best_block, {shape: ms})."""
    p = Params()
    p.dims[:] = [int(d) for d in dims]
    p.block[:] = [2, 2, 2, 2]
    p.m0, p.csw = float(m0), float(csw)
    p.bc[:] = [float(v) for v in bc]
    n = len(candidates) if candidates else 0
    cand = (ctypes.c_int * (4 * n))(*[int(v) for c in candidates for v in c]) if n else None
    out = (ctypes.c_int * 4)()
    times = (ctypes.c_double * (n if n else 64))()
    tried = lib().qcd_tune_block(ctypes.byref(p), _ptr(U), _ptr(b), int(U.is_cuda), ctypes.byref(params) if params else None,
                                 cand, n, ctypes.byref(out), times)
    if tried < 0:
        raise QcdError(tried, "qcd_tune_block")
    shapes = candidates if n else None
    result = {tuple(shapes[i]) if shapes else i: times[i] for i in range(tried)}
    return tuple(out), result


class HmcInfo(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int), ("dH", ctypes.c_double), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
                ("kin0", ctypes.c_double), ("S_g0", ctypes.c_double), ("S_f0", ctypes.c_double),
                ("kin1", ctypes.c_double), ("S_g1", ctypes.c_double), ("S_f1", ctypes.c_double),
                ("solves", ctypes.c_int), ("iterations", ctypes.c_int), ("time_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def qcd_gauge_action(ctx, U, beta):
    S = ctypes.c_double()
    check(lib().qcd_gauge_action(ctx, _ptr(U), ctypes.c_double(beta), ctypes.byref(S), _stream()),
          "qcd_gauge_action")
    return S.value


def qcd_gauge_force(ctx, U, beta, F):
    return check(lib().qcd_gauge_force(ctx, _ptr(U), ctypes.c_double(beta), _ptr(F), _stream()), "qcd_gauge_force")


def qcd_update_links(ctx, U, pi, eps):
    return check(lib().qcd_update_links(ctx, _ptr(U), _ptr(pi), ctypes.c_double(eps), _stream()), "qcd_update_links")


def qcd_hmc_trajectory(ctx, U, pi, eta, beta, eps, nsteps, u_accept, params: SolverParams | None = None):
    info = HmcInfo()
    check(lib().qcd_hmc_trajectory(ctx, _ptr(U), _ptr(pi), _ptr(eta), ctypes.c_double(beta), ctypes.c_double(eps),
                                   int(nsteps), ctypes.c_double(u_accept), ctypes.byref(params) if params else None,
                                   ctypes.byref(info), _stream()), "qcd_hmc_trajectory")
    return info.as_dict()


def qcd_status_string(st):
    return _status_string(st)


def qcd_field_create(ctx, prec="f32"):
    h = ctypes.c_void_p()
    check(lib().qcd_field_create(ctx, PREC[prec], ctypes.byref(h)), "qcd_field_create")
    return h


def qcd_field_create_n(ctx, prec="f32", nrhs=1):
    h = ctypes.c_void_p()
    check(lib().qcd_field_create_n(ctx, PREC[prec], int(nrhs), ctypes.byref(h)), "qcd_field_create_n")
    return h


def qcd_field_free(f):
    lib().qcd_field_free(f)


def qcd_field_import(ctx, f, t):
    return check(lib().qcd_field_import(ctx, f, _ptr(t), _stream()), "qcd_field_import")


def qcd_field_export(ctx, f, t):
    return check(lib().qcd_field_export(ctx, f, _ptr(t), _stream()), "qcd_field_export")


def qcd_apply_D_field(ctx, fin, fout, dagger=False):
    return check(lib().qcd_apply_D_field(ctx, fin, fout, int(dagger), _stream()), "qcd_apply_D_field")


def qcd_apply_D_noalloc(ctx, inp, out, dagger=False):
    """FP64 D (or D^+) without device allocation (lattices up to 65536 sites)."""
    return lib().qcd_apply_D_noalloc(ctx, _ptr(inp), _ptr(out), int(dagger), _stream())


def qcd_sap_apply(ctx, eta, psi, ncy, nmr, prec="f32"):
    return check(lib().qcd_sap_apply(ctx, _ptr(eta), _ptr(psi), int(ncy), int(nmr), PREC[prec], _stream()),
                 "qcd_sap_apply")


def qcd_sap_apply_n(ctx, eta, psi, nrhs, rt, ncy, nmr, prec="f32"):
    """M_SAP on nrhs fields at once, rt right-hand sides per CTA (0: default)."""
    return check(lib().qcd_sap_apply_n(ctx, _ptr(eta), _ptr(psi), int(nrhs), int(rt), int(ncy), int(nmr), PREC[prec],
                                       _stream()), "qcd_sap_apply_n")


def qcd_set_launch(ctx, prec, threads, tps=1):
    """Pin the operator kernel's CTA size and threads per site for one precision."""
    return check(lib().qcd_set_launch(ctx, PREC[prec], int(threads), int(tps)), "qcd_set_launch")


def qcd_get_launch(ctx, prec):
    """(threads, threads per site) of the operator for one precision."""
    t, p = ctypes.c_int(), ctypes.c_int()
    check(lib().qcd_get_launch(ctx, PREC[prec], ctypes.byref(t), ctypes.byref(p)), "qcd_get_launch")
    return t.value, p.value


def qcd_measure_alu_peaks():
    """Measured FMA throughput of this GPU: {"fp32", "fp32x2", "fp64"} in TFLOP/s."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib().qcd_measure_alu_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream()),
          "qcd_measure_alu_peaks")
    return {"fp32": a.value, "fp32x2": b.value, "fp64": c.value}


def qcd_set_sap_tile(ctx, rt):
    return check(lib().qcd_set_sap_tile(ctx, int(rt)), "qcd_set_sap_tile")


def qcd_get_sap_tile(ctx, nrhs):
    rt = lib().qcd_get_sap_tile(ctx, int(nrhs))
    if rt < 0:
        raise QcdError(rt, "qcd_get_sap_tile")
    return rt


DEBUG = {"sap_wait_cycles": 0, "sap_extra_tx": 1}


def qcd_debug_set(ctx, what, value):
    """Test hooks of the SAP staging wait (see include/qcdgb.h)."""
    return check(lib().qcd_debug_set(ctx, DEBUG[what] if isinstance(what, str) else int(what), int(value)),
                 "qcd_debug_set")


def qcd_convert_check(in64, in32, out32, out64):
    """out32 = FP32 of in64 (nearest even), out64 = FP64 of in32, through the
    library's integer-pipe conversions; contiguous CUDA tensors of one length."""
    n = in64.numel()
    assert in32.numel() == n and out32.numel() == n and out64.numel() == n
    return check(lib().qcd_convert_check(_ptr(in64), _ptr(in32), _ptr(out32), _ptr(out64), n, _stream()),
                 "qcd_convert_check")


def qcd_profile_enable(ctx, on=True):
    return check(lib().qcd_profile_enable(ctx, int(on)), "qcd_profile_enable")


def qcd_launch_count():
    return int(lib().qcd_launch_count())


def qcd_profile_reset(ctx):
    return check(lib().qcd_profile_reset(ctx), "qcd_profile_reset")


def qcd_profile_get(ctx, kernel):
    n = ctypes.c_longlong()
    ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    k = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
    check(lib().qcd_profile_get(ctx, k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)),
          "qcd_profile_get")
    return {"launches": n.value, "total_ms": ms.value, "bytes_per_launch": by.value, "flops_per_launch": fl.value}


class Lattice:
    """Convenience owner of one context: dims, Schwarz blocks, action parameters."""

    def __init__(self, dims, block, m0, csw, bc=(-1.0, 1.0, 1.0, 1.0)):
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in block)
        self.m0, self.csw, self.bc = float(m0), float(csw), tuple(bc)
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.ctx = qcd_create(self.dims, self.block, m0, csw, bc)

    def close(self):
        if self.ctx is not None:
            qcd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_gauge(self, U):
        qcd_load_gauge(self.ctx, U)
        qcd_build_clover(self.ctx)

    def apply_D(self, psi, dagger=False, prec="f64"):
        import torch
        out = torch.empty_like(psi)
        nrhs = psi.numel() // (self.V * 12)
        qcd_apply_D(self.ctx, psi.contiguous(), out, dagger, prec, nrhs)
        return out

    def solve(self, b, x0=None, **kw):
        import torch
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        nrhs = b.numel() // (self.V * 12)
        st, info = qcd_solve(self.ctx, b.contiguous(), x, nrhs, solver_params(**kw))
        return x, info

    def hmc_trajectory(self, U, pi, eta, beta, eps, nsteps, u_accept=0.0, **kw):
        """One HMC trajectory; U (V,4,3,3) complex128 and pi (V,4,8) float64 device
        tensors are updated in place."""
        return qcd_hmc_trajectory(self.ctx, U, pi, eta, beta, eps, nsteps, u_accept, solver_params(**kw))

    def sap(self, eta, ncy=4, nmr=4, prec="f32"):
        import torch
        psi = torch.empty_like(eta)
        qcd_sap_apply(self.ctx, eta.contiguous(), psi, ncy, nmr, prec)
        return psi
