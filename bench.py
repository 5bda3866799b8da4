#!/usr/bin/env python3
"""Benchmark: SAP+FGCR time to |r|/|b| < 1e-10 and D_w GB/s on one GB300.

Workload: 32^3 x 64 lattice, links exp(i 0.5 sum_a g_a lambda_a / 2) (seed 3),
m0 = -0.05, c_sw = 1.5, antiperiodic time; one complex Gaussian right-hand
side; SAP (4 MR steps, 4 cycles; block shape 4^4 or 8x4x4x4 chosen by the
autotuner) with FP16 block fields and FP32 arithmetic; FGCR(16) whose
recursion (outer operator, Gram-Schmidt, dots, updates) runs in double-float
arithmetic on the FP32 units (--outer-prec df64, the default; f64 runs it in
native FP64), with the solution in FP64 and the restart residual r = b - D x
formed in FP64 from a double-float D x.  A step is one complete solve from
x = 0 to a true residual <= 1e-10.

Every vector of the solve (403 MB each in FP64) and the gauge/clover fields
exceed the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The reference arm times the plain FP64 CPU oracle (oracle/) on the host cores:
each step is one SAP-FGCR iteration of the same solve, extrapolated by the
iteration count the GPU solve needs.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "32^3x64_fp16"
# the benchmarked solve, and a smaller lattice of the same recipe whose
# working set still exceeds L2 (used for detailed profiler captures)
BENCH_WORKLOADS = {
    "32^3x64_fp16": dict(dims=(64, 32, 32, 32), eps=0.5, seed=3, m0=-0.05, csw=1.5, block=(4, 4, 4, 4),
                         nmr=4, ncy=4, nkv=16),
    "24^3x48_fp16": dict(dims=(48, 24, 24, 24), eps=0.5, seed=4, m0=-0.05, csw=1.5, block=(4, 4, 4, 4),
                         nmr=4, ncy=4, nkv=16),
}
METRIC = "SAP+FGCR time to |r|/|b|<1e-10 and D_w GB/s vs HBM peak, 1 GB300"
# algorithmic bytes per site of one operator apply: spinor in + out, 4 links
# as 12 reals (two rows), 72-real clover; 16-bit adds the per-site scales
DW_BYTES = {"f64": 1344.0, "f32": 672.0, "f16": 352.0}
DW_FLOPS = 1824.0  # 1320 hopping + 504 clover per site
# DRAM bytes (read + write) per solved site of one FP16 SAP launch, averaged over
# the 8 launches of one preconditioner application (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, 24^3x48 lattice, 331,776 solved sites per launch); valid
# for the kernel sources whose hash is stored with it and that block shape,
# scaled by solved sites
SAP_TRAFFIC = {"bytes_per_site": 572.6, "src_sha": "06e92ebc34f7c7a3", "block": (8, 4, 4, 4)}


def sap_src_sha():
    h = hashlib.sha256()
    for f in ("sap.cu", "qcd.cuh"):
        with open(os.path.join(ROOT, "paper_1109_4279_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]
DTYPE = {(sp, op): "%s recursion (f64 solution; f64 restart residual, its D x in df64 with the df64 recursion) + %s SAP arithmetic on %s SAP storage"
                   % ({"df64": "df64 (double-float: FP32 pairs with error-free transforms, chi = D phi included)"}.get(op, op),
                      "f64" if sp == "f64" else "f32", sp)
         for sp in ("f64", "f32", "f16", "bf16") for op in ("f64", "f32", "df64")}


def peaks(measure=True):
    """Roofline denominators.  HBM: the measured copy rate
    (MEASURED_PEAKS.json; 6.8 TB/s fallback).  FP32 / FP64: fused multiply-add
    throughput measured on this GPU by qcd_measure_alu_peaks (the larger of
    scalar FP32 and packed FP32x2), next to the unit-count figures (SM count
    read from the device, 128 FP32 and 2 FP64 lanes per SM, maximum clock)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    p = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        p.update({k: d[k] for k in ("hbm_gbs", "sm_max_mhz") if k in d})
        p["source"] = "measured"
    mhz = p["sm_max_mhz"]
    sms = 152
    try:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:
        pass
    p["sms"] = sms
    p["fp32_tflops_units"] = sms * 128 * 2 * mhz * 1e6 / 1e12
    p["fp64_tflops_units"] = sms * 2 * 2 * mhz * 1e6 / 1e12
    p["fp32_tflops"], p["fp64_tflops"], p["alu_source"] = p["fp32_tflops_units"], p["fp64_tflops_units"], "units"
    if measure:
        from paper_1109_4279_gb300 import binding as B
        m = B.qcd_measure_alu_peaks()
        p["alu_measured"] = m
        p["fp32_tflops"] = max(m["fp32"], m["fp32x2"])
        p["fp64_tflops"] = m["fp64"]
        p["alu_source"] = "measured (qcd_measure_alu_peaks)"
    return p


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region: sampling
    every 50 ms starts before the region (the first sample is awaited), and
    only samples stamped inside the region are summarised (all of them if
    none is)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        import datetime
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "50"]
        if self.uuid:
            cmd[1:1] = ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        deadline = time.time() + 3.0
        while self.proc is not None and time.time() < deadline and os.path.getsize(self.path) == 0:
            time.sleep(0.01)
        self.t0 = datetime.datetime.now()
        return self

    def __exit__(self, *exc):
        import datetime
        self.t1 = datetime.datetime.now()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                    rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 is not None and self.t1 is not None and self.t0 <= r[0] <= self.t1]
        use = inside or rows
        if use:
            reasons = sorted({name for r in use for name, val in zip(names, r[3]) if val.lower().startswith("active")})
            out.update(sm_mhz=statistics.median(r[1] for r in use), sm_max_mhz=max(r[2] for r in use),
                       reasons=reasons, samples=len(use), in_timed_region=bool(inside))
        return out


def make_inputs(workload=WORKLOAD):
    from paper_1109_4279_gb300 import synth
    w = BENCH_WORKLOADS[workload]
    U, rng = synth.gauge_field(w["dims"], w["eps"], w["seed"])
    b = synth.gaussian_spinor(w["dims"], rng)
    return w, U, b


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value, device="cuda"):
    """Largest value over all ranks (the slowest rank's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def from_rank0(world, value, device="cuda"):
    """rank 0's integer value on every rank (one choice for all replicas)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(value)], dtype=torch.int64, device=device)
    dist.broadcast(t, src=0)
    return int(t.item())


# --------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# --------------------------------------------------------------------------
def oracle_iteration_seconds(w, U, b):
    """One SAP-FGCR iteration of the oracle on the full lattice (all host cores)."""
    import oracle
    oracle.build()
    A = oracle.clover(w["dims"], U, w["m0"], w["csw"])
    from paper_1109_4279_gb300 import synth
    t0 = time.perf_counter()
    oracle.fgcr(w["dims"], U, A, synth.ANTIPERIODIC_T, b, nkv=w["nkv"], max_restarts=1, tol=1e-10, precond=True,
                block=w["block"], ncy=w["ncy"], nmr=w["nmr"], max_iters=1)
    return time.perf_counter() - t0, oracle.num_threads()


# the Schwarz block shape the autotuner picks on these workloads (complete
# solves on 32^3x64 with the double-float recursion: 8x4x4x4 44.3 ms against
# 4^4 47.4 ms) and the iteration count with it (6, as with the FP64
# recursion); the oracle legs run the same method
REFERENCE_BLOCK = (8, 4, 4, 4)


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    w, U, b = make_inputs(args.workload)
    w = dict(w, block=REFERENCE_BLOCK)
    iters = args.gpu_iterations
    times = []
    threads = 0
    for k in range(args.warmup + args.steps):
        t, threads = oracle_iteration_seconds(w, U, b)
        if k >= args.warmup:
            times.append(t)
    t_iter = statistics.median(times)
    value = t_iter * iters
    sample = ("one SAP-FGCR iteration of the oracle on the full %s lattice per step (clover build not "
              "timed), extrapolated x%d iterations (the FP64 recursion's count on this workload, "
              "measured on the GPU)" % (args.workload.split()[0], iters))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_iter * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "dims": list(w["dims"]), "block": list(w["block"]), "m0": w["m0"],
                       "csw": w["csw"], "eps": w["eps"], "seed": w["seed"], "tol": 1e-10, "nkv": w["nkv"],
                       "ncy": w["ncy"], "nmr": w["nmr"], "sap_prec": "f64 (oracle)", "outer_prec": "f64"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def time_dirac(lat, b_t, prec, reps=20, nrhs=1):
    """Resident-field operator apply (nrhs right-hand sides per launch): ms per launch."""
    import torch
    from paper_1109_4279_gb300 import binding as B
    fi = B.qcd_field_create_n(lat.ctx, prec, nrhs)
    fo = B.qcd_field_create_n(lat.ctx, prec, nrhs)
    B.qcd_field_import(lat.ctx, fi, b_t.expand(nrhs, *b_t.shape).contiguous() if nrhs > 1 else b_t)
    for _ in range(3):
        B.qcd_apply_D_field(lat.ctx, fi, fo)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        B.qcd_apply_D_field(lat.ctx, fi, fo)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    B.qcd_field_free(fi)
    B.qcd_field_free(fo)
    return ms


def _time_solve(lat, b_t, sp, reps=1):
    """Median device time (ms) of complete solves from x = 0 after one warm-up."""
    import torch
    from paper_1109_4279_gb300 import binding as B
    x = torch.zeros_like(b_t)
    spz = B.SolverParams.from_buffer_copy(sp)
    spz.zero_guess = 1  # x = 0 through the API, as in the timed solves
    times, info = [], None
    for k in range(reps + 1):
        st, inf = B.qcd_solve(lat.ctx, b_t, x, 1, spz, raise_on_fail=False)
        info = inf[0]
        if k:
            times.append(info["time_ms"])
    return statistics.median(times), info


def run_comparisons(args, lat, w, U, b_t, sp_main, main_ms):
    """Time-to-solution of the same system with other precision splits, the
    deflated-restart solver and the plain FP64 solvers (one timed solve each
    after a warm-up).  A variant whose block fields do not fit in shared memory
    with the benchmarked block shape (FP32 SAP fields of 8x4x4x4 blocks) runs
    with 4^4 blocks; all-FP64 SAP with 4x4x4x2 blocks; each entry names its
    block shape."""
    import torch
    from paper_1109_4279_gb300 import binding as B
    main = "sap_%s_outer_%s" % (args.sap_prec, args.outer_prec)
    blk = "x".join(map(str, w["block"]))
    out = {main: {"ms": main_ms, "block": blk, "note": "the benchmarked solve"}}
    lats = {tuple(w["block"]): lat}

    def lattice(block):
        if block not in lats:
            lats[block] = B.Lattice(w["dims"], block, w["m0"], w["csw"])
            lats[block].load_gauge(torch.from_numpy(U).cuda())
        return lats[block]

    variants = [("sap_%s_outer_%s" % (sp_, op_), dict(sap_prec=sp_, outer_prec=op_))
                for sp_, op_ in (("f16", "f64"), ("f16", "df64"), ("bf16", "df64"), ("f16", "f32"), ("f32", "f32"),
                                 ("bf16", "f32"), ("f32", "f64"), ("f64", "f64"))]
    # the double-float recursion with its restart residual entirely in FP64
    variants.append(("sap_f16_outer_df64_residual_f64", dict(sap_prec="f16", outer_prec="df64", residual_prec="f64")))
    variants.append(("fgmres_dr_16_4_sap_f16_outer_f64", dict(solver="fgmres_dr", ndefl=4, sap_prec="f16")))
    variants.append(("gcr_f64_unpreconditioned", dict(precond="none", max_restarts=400)))
    variants.append(("cgne_f64", dict(solver="cg")))
    variants.append(("cg_eo_f64", dict(solver="cg_eo")))
    for name, kw in variants:
        if name == main:
            continue
        sp = B.solver_params(tol=1e-10, nkv=w["nkv"], ncy=w["ncy"], nmr=w["nmr"], **kw)
        for block in (tuple(w["block"]), (4, 4, 4, 4), (4, 4, 4, 2)):
            ms, info = _time_solve(lattice(block), b_t, sp)
            if info["status"] != -11:  # QCD_ERR_UNSUPPORTED: block fields exceed shared memory
                break
        out[name] = {"ms": ms, "block": "x".join(map(str, block)),
                     "iterations": info["cg_iterations"] if kw.get("solver") in ("cg", "cg_eo") else info["iterations"],
                     "status": info["status"], "true_residual": info["true_residual"]}
    for block, l in lats.items():
        if l is not lat:
            l.close()
    # the fastest plain FP64 solve: all-FP64 SAP-FGCR, unpreconditioned GCR, CG on D^+ D, even/odd CG
    plain = min(out[k]["ms"] for k in ("gcr_f64_unpreconditioned", "sap_f64_outer_f64", "cgne_f64", "cg_eo_f64"))
    out["speedup_vs_plain_fp64"] = plain / main_ms
    return out


def run_near_critical(args):
    """Sec. 4 Fig. 1 analogue: 16^3 x 32 (eps 0.5, seed 2, c_sw 1.5) at
    m0 = -0.45, close to the critical mass of this ensemble: FGCR with plain
    restarts of 8 and 16 vectors against FGMRES-DR with 4 deflated vectors."""
    import numpy as np
    import torch
    from paper_1109_4279_gb300 import binding as B, synth
    dims = (32, 16, 16, 16)
    U, rng = synth.gauge_field(dims, 0.5, 2)
    b = torch.from_numpy(synth.gaussian_spinor(dims, rng)).cuda()
    lat = B.Lattice(dims, (4, 4, 4, 4), -0.45, 1.5)
    lat.load_gauge(torch.from_numpy(U).cuda())
    out = {"workload": "16^3x32, m0 -0.45, SAP f16 (4 cycles, 4 MR), FP64 recursion, tol 1e-10"}
    for name, kw in (("fgcr_8", dict(nkv=8)), ("fgcr_16", dict(nkv=16)),
                     ("fgmres_dr_8_4", dict(nkv=8, solver="fgmres_dr", ndefl=4)),
                     ("fgmres_dr_16_4", dict(nkv=16, solver="fgmres_dr", ndefl=4))):
        sp = B.solver_params(tol=1e-10, sap_prec="f16", max_restarts=400, **kw)
        ms, info = _time_solve(lat, b, sp)
        out[name] = {"ms": ms, "iterations": info["iterations"], "cycles": info["restarts"],
                     "status": info["status"], "true_residual": info["true_residual"]}
    lat.close()
    return out


def run_configs(args, pk):
    """The other named workloads, one measurement each (CUDA events / wall
    clock around complete calls with synchronisation; setup not timed)."""
    import numpy as np
    import torch
    from paper_1109_4279_gb300 import binding as B, synth
    out = {}
    # 4^4, FP64 throughout (SAP on 2^4 blocks with FP64 fields)
    wl = synth.WORKLOADS["4^4 fp64"]
    U, rng = synth.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    b = torch.from_numpy(synth.gaussian_spinor(wl["dims"], rng)).cuda()
    lat = B.Lattice(wl["dims"], wl["block"], wl["m0"], wl["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    ms, info = _time_solve(lat, b, B.solver_params(tol=1e-10, sap_prec="f64"))
    out["4^4_fp64_solve"] = {"ms": ms, "iterations": info["iterations"], "true_residual": info["true_residual"]}
    lat.close()
    # 16^3 x 32: operator apply in FP64 and FP32 (fields of 100 / 50 MB: L2-resident), FP32-SAP solve
    wl = synth.WORKLOADS["16^3x32 fp32"]
    V = int(np.prod(wl["dims"]))
    U, rng = synth.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    bn = synth.gaussian_spinor(wl["dims"], rng)
    b = torch.from_numpy(bn).cuda()
    lat = B.Lattice(wl["dims"], wl["block"], wl["m0"], wl["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    for prec in ("f64", "f32"):
        ms = time_dirac(lat, b, prec, reps=50)
        out["16^3x32_dw_" + prec] = {"ms": ms, "gbs": DW_BYTES[prec] * V / (ms * 1e-3) / 1e9,
                                     "gflops": DW_FLOPS * V / (ms * 1e-3) / 1e9, "note": "fields L2-resident"}
    ms, info = _time_solve(lat, b, B.solver_params(tol=1e-10, sap_prec="f32"))
    out["16^3x32_sap_f32_solve"] = {"ms": ms, "iterations": info["iterations"], "true_residual": info["true_residual"]}
    lat.close()
    # ten uneven lattices in one batched call against one at a time
    blocks = {(8, 8, 8, 8): (4, 4, 2, 2), (16, 8, 8, 8): (4, 4, 4, 4), (24, 12, 12, 12): (4, 6, 2, 2),
              (32, 16, 16, 16): (4, 4, 4, 4)}
    lats, bs, xs = [], [], []
    for k, dims in enumerate(synth.UNEVEN_LATTICES):
        U, rng = synth.gauge_field(dims, 0.5, 10 + k)
        l = B.Lattice(dims, blocks[dims], 0.0, 1.5)
        l.load_gauge(torch.from_numpy(U).cuda())
        lats.append(l)
        bs.append(torch.from_numpy(synth.gaussian_spinor(dims, rng)).cuda())
        xs.append(torch.zeros_like(bs[-1]))
    sp = B.solver_params(tol=1e-10, sap_prec="f16")
    for _ in range(2):  # warm-up (workspaces, graphs), then timed
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, infos = B.qcd_solve_batch([l.ctx for l in lats], bs, xs, sp)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
    t_seq = 0.0
    for l, bb, x in zip(lats, bs, xs):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.qcd_solve(l.ctx, bb, x, 1, sp)
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
    out["uneven_10_lattices"] = {"batched_s": t_batch, "sequential_s": t_seq,
                                 "max_true_residual": max(i["true_residual"] for i in infos)}
    for l in lats:
        l.close()
    # 16^3 x 32 gradient: solve, adjoint solve (gamma5 D gamma5) and force
    wl = synth.WORKLOADS["16^3x32 gradient"]
    U, rng = synth.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    phi = torch.from_numpy(synth.gaussian_spinor(wl["dims"], rng)).cuda()
    lat = B.Lattice(wl["dims"], wl["block"], wl["m0"], wl["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    V = int(np.prod(wl["dims"]))
    dphi = torch.empty_like(phi)
    dth = torch.empty((V, 4, 8), dtype=torch.float64, device="cuda")
    sp = B.solver_params(tol=1e-10, sap_prec="f16")
    for k in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.qcd_gradient(lat.ctx, phi, dphi, dth, None, None, sp)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - t0
    out["16^3x32_gradient"] = {"s": t_grad, "note": "x = D^-1 phi, y = gamma5 D^-1 gamma5 phi, dL/dphi and the "
                                                    "su(3) force of every link"}
    # one HMC trajectory on the same lattice: beta 5.5, 5 leapfrog steps of 0.02,
    # two clover flavours (2 solves per force, 1 per Hamiltonian)
    pi = torch.from_numpy(rng.standard_normal((V, 4, 8))).cuda()
    eta = torch.from_numpy(synth.gaussian_spinor(wl["dims"], rng)).cuda()
    Ud = torch.from_numpy(U.copy()).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = lat.hmc_trajectory(Ud, pi, eta, 5.5, 0.02, 5, 0.0, tol=1e-10, sap_prec="f16")
    torch.cuda.synchronize()
    out["16^3x32_hmc_trajectory"] = {"s": time.perf_counter() - t0, "dH": info["dH"], "solves": info["solves"],
                                     "iterations": info["iterations"], "accepted": info["accepted"],
                                     "note": "beta 5.5, 5 leapfrog steps of 0.02, FP16 SAP, tol 1e-10"}
    lat.close()
    return out


def run_batched(args, block):
    """12 spin-colour point sources on 24^3 x 48 (eps 0.5, seed 4, m0 0,
    c_sw 1.5), with the Schwarz block shape of the main solve: one
    multi-right-hand-side call (every launch of an FGCR iteration runs over
    all twelve; the SAP tile chosen by the autotuner) against 12 single
    solves."""
    import numpy as np
    import torch
    from paper_1109_4279_gb300 import binding as B, synth
    wl = synth.WORKLOADS["24^3x48 12 point sources"]
    U, _ = synth.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    b = torch.from_numpy(synth.point_sources(wl["dims"])).cuda()
    lat = B.Lattice(wl["dims"], block, wl["m0"], wl["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    B.qcd_autotune(lat.ctx, 12)
    rt = B.qcd_get_sap_tile(lat.ctx, 12)
    sp = B.solver_params(tol=1e-10, nkv=wl["nkv"], ncy=wl["ncy"], nmr=wl["nmr"], sap_prec=args.sap_prec,
                         outer_prec=args.outer_prec)
    x = torch.zeros_like(b)
    for _ in range(2):  # warm-up (workspaces, graph capture), then timed
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = B.qcd_solve(lat.ctx, b, x, 12, sp)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
    t_seq = 0.0
    for k in range(12):
        xk = torch.zeros_like(b[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.qcd_solve(lat.ctx, b[k].contiguous(), xk, 1, sp)
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
    lat.close()
    return {"workload": "24^3x48, 12 point sources, SAP %s / FGCR %s, blocks %s" % (
                args.sap_prec, args.outer_prec, "x".join(map(str, block))),
            "sap_rhs_tile": rt, "batched_s": t_batch, "sequential_s": t_seq, "speedup": t_seq / t_batch,
            "solves_per_s_batched": 12 / t_batch, "solves_per_s_sequential": 12 / t_seq,
            "iterations": [i["iterations"] for i in info], "max_true_residual": max(i["true_residual"] for i in info)}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1109_4279_gb300 import binding as B

    pk = peaks()
    w, U, b = make_inputs(args.workload)
    V = int(np.prod(w["dims"]))
    w = dict(w)
    tuning = None
    if args.block:
        w["block"] = tuple(int(v) for v in args.block.split("x"))
    elif not args.no_tune:
        # Schwarz block shape by the autotuner (timed complete solves, outside
        # the timed region): 4^4 against 8 x 4^3 (8 along time)
        cands = [c for c in ((4, 4, 4, 4), (8, 4, 4, 4))
                 if all(w["dims"][m] % c[m] == 0 and (w["dims"][m] // c[m]) % 2 == 0 for m in range(4))]
        sp_t = B.solver_params(tol=1e-10, nkv=w["nkv"], ncy=w["ncy"], nmr=w["nmr"], sap_prec=args.sap_prec,
                               outer_prec=args.outer_prec)
        best, times = B.qcd_tune_block(w["dims"], w["m0"], w["csw"], torch.from_numpy(U).cuda(),
                                       torch.from_numpy(b).cuda(), candidates=cands, params=sp_t)
        # every replica runs rank 0's choice
        w["block"] = cands[from_rank0(world, cands.index(tuple(best)))]
        tuning = {"x".join(map(str, c)): t for c, t in times.items()}
    lat = B.Lattice(w["dims"], w["block"], w["m0"], w["csw"])
    lat.load_gauge(torch.from_numpy(U).cuda())
    B.qcd_autotune(lat.ctx, 1)  # operator launch shapes, outside the timed region
    launch = {p: B.qcd_get_launch(lat.ctx, p) for p in ("f64", "f32", "f16", "df64")}
    b_t = torch.from_numpy(b).cuda()
    x_t = torch.zeros_like(b_t)
    sp = B.solver_params(tol=1e-10, nkv=w["nkv"], ncy=w["ncy"], nmr=w["nmr"], sap_prec=args.sap_prec,
                         outer_prec=args.outer_prec)
    # x = 0 as the initial guess, stated through the API (zero_guess): the
    # solver neither reads x nor needs it cleared; every step writes it anew
    sp_step = B.SolverParams.from_buffer_copy(sp)
    sp_step.zero_guess = 1

    def solve_once():
        st, info = B.qcd_solve(lat.ctx, b_t, x_t, 1, sp_step)
        return info[0]

    for _ in range(args.warmup):
        solve_once()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None

    B.qcd_profile_reset(lat.ctx)
    B.qcd_profile_enable(lat.ctx, True)
    launches0 = B.qcd_launch_count()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(solve_once())
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = B.qcd_launch_count() - launches0
    B.qcd_profile_enable(lat.ctx, False)
    elapsed_ms = max_over_ranks(world, e0.elapsed_time(e1))
    ms_per_step = elapsed_ms / args.steps
    for inf in infos:
        assert inf["status"] == 0 and inf["true_residual"] <= 1e-10, inf
    iters = int(statistics.median(i["iterations"] for i in infos))

    kernels = {}
    for name in ("sap", "dirac", "blas", "residual"):
        p = B.qcd_profile_get(lat.ctx, name)
        if p["launches"]:
            avg = p["total_ms"] / p["launches"]
            kernels[name] = {"launches": p["launches"], "total_ms": p["total_ms"], "avg_ms": avg,
                             "share": p["total_ms"] / elapsed_ms,
                             "achieved_tflops": p["flops_per_launch"] / (avg * 1e-3) / 1e12,
                             "achieved_gbs": p["bytes_per_launch"] / (avg * 1e-3) / 1e9}
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    kd = kernels[dom]
    if dom == "sap":
        roof = {"kernel": "sap_sweep (%s block fields, %s arithmetic)" % (args.sap_prec.upper(),
                                                                         "FP64" if args.sap_prec == "f64" else "FP32"),
                "bound": "alu",
                "achieved": kd["achieved_tflops"], "peak": pk["fp32_tflops"], "unit": "TFLOP/s"}
    elif dom in ("dirac", "residual"):
        roof = {"kernel": "dirac FP64", "bound": "alu", "achieved": kd["achieved_tflops"],
                "peak": pk["fp64_tflops"], "unit": "TFLOP/s"}
    else:
        roof = {"kernel": "blas FP64", "bound": "hbm", "achieved": kd["achieved_gbs"], "peak": pk["hbm_gbs"],
                "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    if (dom == "sap" and args.sap_prec == "f16" and SAP_TRAFFIC["bytes_per_site"]
            and SAP_TRAFFIC["src_sha"] == sap_src_sha() and tuple(w["block"]) == SAP_TRAFFIC["block"]):
        roof["traffic"] = SAP_TRAFFIC["bytes_per_site"] * V / 2
    roof["peak_source"] = ("FP32/FP64: %s on this GPU (unit counts at %.0f MHz: %.1f / %.2f TFLOP/s); "
                           "HBM: MEASURED_PEAKS.json" % (pk["alu_source"], pk["sm_max_mhz"], pk["fp32_tflops_units"],
                                                         pk["fp64_tflops_units"]))

    # D_w bandwidth per precision (resident fields)
    dw = {}
    for prec in ("f64", "f32", "f16"):
        ms = time_dirac(lat, b_t, prec)
        gbs = DW_BYTES[prec] * V / (ms * 1e-3) / 1e9
        dw[prec] = {"ms": ms, "gbs": gbs, "frac_hbm_measured": gbs / pk["hbm_gbs"], "frac_hbm_nominal_8tbs": gbs / 8000.0,
                    "gflops": DW_FLOPS * V / (ms * 1e-3) / 1e9}

    # multi-right-hand-side operator: links and clover read once per site for R
    # fields, CTA sizes tuned for R right-hand sides
    R = 12
    B.qcd_autotune(lat.ctx, R)
    for prec in ("f32", "f16"):
        ms = time_dirac(lat, b_t, prec, reps=10, nrhs=R)
        spin = {"f32": 192.0, "f16": 104.0}[prec]
        byts = (DW_BYTES[prec] - spin + spin * R) * V
        gbs = byts / (ms * 1e-3) / 1e9
        dw[prec + "_x%d_rhs" % R] = {"ms": ms, "gbs": gbs, "frac_hbm_measured": gbs / pk["hbm_gbs"],
                                     "bytes_per_site_rhs": byts / V / R,
                                     "site_rhs_per_s": V * R / (ms * 1e-3),
                                     "launch": B.qcd_get_launch(lat.ctx, prec)}

    B.qcd_autotune(lat.ctx, 1)  # back to the single-right-hand-side shapes of the timed solve
    # the operator kernels' rooflines next to the dominant kernel's
    roof["operators"] = {k: {"ms": v["ms"], "gbs": v["gbs"], "frac_hbm": v["frac_hbm_measured"]}
                         for k, v in dw.items()}
    roof["operators"]["f64"]["bound"] = "fp64 alu"
    roof["operators"]["f64"]["frac_fp64_alu"] = dw["f64"]["gflops"] / 1e3 / pk["fp64_tflops"]

    # the comparison sections run at N = 1 only (they hold the GPUs for minutes)
    extra = not args.quick and world == 1
    comparisons = run_comparisons(args, lat, w, U, b_t, sp, ms_per_step) if extra else None
    batched = run_batched(args, tuple(w["block"])) if extra else None
    near_critical = run_near_critical(args) if extra else None
    configs = run_configs(args, pk) if extra else None

    # end to end through the public API with host buffers
    b_h = torch.from_numpy(b.copy()).pin_memory()
    x_h = torch.empty_like(b_h).pin_memory()
    # x = 0 as the initial guess, stated through the API (zero_guess): the
    # step's only input is b, and x is only written back
    sp_e2e = B.SolverParams.from_buffer_copy(sp)
    sp_e2e.zero_guess = 1
    e2e_times = []
    # at least 7 samples: single host-buffer solves occasionally take tens of
    # milliseconds longer on the host side, and the median must not see them
    for k in range(max(args.steps, 7) + 1):
        x_h.fill_(float("nan"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = B.qcd_solve(lat.ctx, b_h, x_h, 1, sp_e2e)
        torch.cuda.synchronize()
        if k:
            e2e_times.append(time.perf_counter() - t0)
        assert st == 0
    e2e_s = max_over_ranks(world, statistics.median(e2e_times))
    fbytes = V * 12 * 16

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_iter, threads = oracle_iteration_seconds(w, U, b)
        n_or = iters
        cpu = {"value": t_iter * n_or, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": "one SAP-FGCR iteration of the FP64 oracle on the full %s lattice with %s blocks "
                         "(%.1f s), extrapolated x%d iterations (the GPU solve's count with these blocks)"
                         % (args.workload.split()[0], "x".join(map(str, w["block"])), t_iter, n_or)}

    line = {"metric": METRIC, "value": ms_per_step / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[(args.sap_prec, args.outer_prec)], "data": "synthetic",
            "config": {"workload": args.workload, "dims": list(w["dims"]), "block": list(w["block"]), "m0": w["m0"],
                       "csw": w["csw"], "eps": w["eps"], "seed": w["seed"], "tol": 1e-10, "nkv": w["nkv"],
                       "ncy": w["ncy"], "nmr": w["nmr"], "sap_prec": args.sap_prec, "outer_prec": args.outer_prec,
                       "iterations": iters, "restarts": int(statistics.median(i["restarts"] for i in infos)),
                       "true_residual": max(i["true_residual"] for i in infos),
                       "l2": "no flush: every FP64 solver vector (192 B/site) and the gauge/clover fields exceed the 129 MB L2",
                       "block_tuning_ms": tuning,
                       "operator_launch": {p: {"threads": t, "threads_per_site": q} for p, (t, q) in launch.items()}},
            "roofline": roof, "kernels": kernels, "dw": dw, "comparisons": comparisons, "batched": batched,
            "near_critical": near_critical, "configs": configs,
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": fbytes, "d2h_bytes_per_step": fbytes},
            "gpu_launches": launches,
            "clocks": clk.summary(), "cpu_baseline": cpu,
            "peaks": {"hbm_gbs": pk["hbm_gbs"], "fp32_tflops": pk["fp32_tflops"], "fp64_tflops": pk["fp64_tflops"],
                      "source": pk["source"], "alu_source": pk["alu_source"], "alu_measured": pk.get("alu_measured"),
                      "sms": pk["sms"]}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(BENCH_WORKLOADS), default=WORKLOAD)
    ap.add_argument("--gpu-iterations", type=int, default=6,
                    help="reference arm: FGCR iterations of the FP64 recursion on this workload with "
                         "8x4x4x4 blocks (measured on the GPU: 6)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the comparison and batched sections")
    ap.add_argument("--no-tune", action="store_true", help="use the workload's 4^4 blocks without the block autotuner")
    ap.add_argument("--block", default=None, help="Schwarz block shape, e.g. 8x4x4x4 (skips the autotuner)")
    ap.add_argument("--sap-prec", choices=["f64", "f32", "f16", "bf16"], default="f16",
                    help="storage precision of the SAP block fields")
    ap.add_argument("--outer-prec", choices=["f64", "df64", "f32"], default="df64",
                    help="FGCR recursion precision: f64 (Gram-Schmidt, dots, chi = D phi and the update in FP64), "
                         "df64 (the same recursion, chi = D phi included, in double-float arithmetic on the FP32 "
                         "units; FP64 solution, restart residual b - D x in FP64 with D x in double-float) or f32 (the paper's iterative-refinement split, FP64 only "
                         "at restarts)")
    args = ap.parse_args()
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        return run_reference(args, world, rank)
    world, rank, local = dist_setup()
    rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
