"""Timings of the FP64 oracle on the host cores: the CPU baseline beside the
GPU numbers (test infrastructure; nothing in the library uses it).

  * the operator D on the 16^3 x 32 and 32^3 x 64 workloads, best of 5;
  * unpreconditioned GCR(16) to |r|/|b| <= 1e-10 on the 4^4 and 16^3 x 32
    workloads;
  * on 32^3 x 64 the time of 8 GCR iterations, scaled to the iteration count
    the GPU's FP64 GCR needs there (an estimate, labelled as one).

The thread count is OpenMP's (OMP_NUM_THREADS); one JSON line per timing:

  OMP_NUM_THREADS=1 python -m oracle.timing
  python -m oracle.timing
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GPU_GCR_ITERATIONS_32x64 = 107  # the GPU's unpreconditioned FP64 GCR(16) on 32^3 x 64 to 1e-10


def _workload(name):
    from paper_1109_4279_gb300 import synth
    w = synth.WORKLOADS[name]
    U, rng = synth.gauge_field(w["dims"], w["eps"], w["seed"])
    b = synth.gaussian_spinor(w["dims"], rng)
    return w, U, b


def main():
    import oracle
    from paper_1109_4279_gb300 import synth
    oracle.build()
    threads = oracle.num_threads()
    bc = synth.ANTIPERIODIC_T
    out = []

    def emit(**kw):
        kw["threads"] = threads
        print(json.dumps(kw), flush=True)
        out.append(kw)

    for name in ("16^3x32 fp32", "32^3x64 fp16"):
        w, U, b = _workload(name)
        A = oracle.clover(w["dims"], U, w["m0"], w["csw"])
        best = float("inf")
        for _ in range(5):
            t0 = time.perf_counter()
            oracle.apply_D(w["dims"], U, A, bc, b)
            best = min(best, time.perf_counter() - t0)
        emit(what="D apply, best of 5", workload=name, seconds=best)
        if name == "32^3x64 fp16":
            t0 = time.perf_counter()
            _, it, _, _, _ = oracle.fgcr(w["dims"], U, A, bc, b, nkv=16, tol=1e-10, max_iters=8)
            t = (time.perf_counter() - t0) / max(it, 1)
            emit(what="GCR(16) solve to 1e-10, estimate", workload=name, seconds_per_iteration=t,
                 iterations=GPU_GCR_ITERATIONS_32x64, seconds=t * GPU_GCR_ITERATIONS_32x64)
    for name in ("4^4 fp64", "16^3x32 fp32"):
        w, U, b = _workload(name)
        A = oracle.clover(w["dims"], U, w["m0"], w["csw"])
        t0 = time.perf_counter()
        _, it, cy, conv, res = oracle.fgcr(w["dims"], U, A, bc, b, nkv=16, max_restarts=1000, tol=1e-10)
        emit(what="GCR(16) solve to 1e-10", workload=name, seconds=time.perf_counter() - t0, iterations=it,
             converged=conv, true_rel_res=res)
    return out


if __name__ == "__main__":
    main()
