// Flexible GCR with restarts, preconditioned by the Schwarz alternating
// procedure, in mixed precision (Sec. 4).  The recursion (Gram-Schmidt,
// global dot products, solution update) and the true residual at every
// restart are FP64; the preconditioner runs on reduced-precision block fields.
//
// Iteration k of a cycle (rho_0 = r = b - D x):
//   phi_k = M_SAP rho_k;  chi_k = D phi_k;
//   chi_k -= sum_j a_jk chi_j   (classical Gram-Schmidt; a second pass when
//                                the first cancelled more than half the norm);
//   chi_k /= |chi_k|;  c_k = (chi_k, rho_k);  rho_{k+1} = rho_k - c_k chi_k.
// At the end of a cycle the upper-triangular system H gamma = c is solved on
// the device, x += sum_k gamma_k phi_k, and r = b - D x is recomputed in FP64.
//
// Two precisions of the recursion:
//  - FP64 (outer_prec = F64): rho, phi_k, chi_k and every dot product in FP64;
//  - FP32 (outer_prec = F32), the scheme of Sec. 4 (iterative refinement):
//    every operation of a cycle is single precision, on the normalised
//    residual rho_0 = r / |r|; the cycle ends when |rho_k| has dropped by
//    inner_tol (or below the target); then the FP32 correction
//    |r| sum_k gamma_k phi_k is added to the FP64 solution and the residue is
//    recomputed in double precision.
//
// Many right-hand sides or lattices (Sec. 4: flexibility in the lattice
// sizes) are solved in lock step: every iteration is enqueued for all active
// problems, each on its own stream and workspace, so their kernels run
// concurrently, and one host synchronisation per iteration reads all the
// recursive residuals.  With use_graphs each problem's iteration k is captured
// once as a CUDA graph and replayed (one launch instead of ~20).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace qcd {

size_t partials_for(long long V) {
  const size_t blas = (size_t)152 * 8 * 65;     // largest BLAS grid x widest record
  const size_t resid = (size_t)(V + 255) / 256;  // one partial per residual CTA
  return blas > resid ? blas : resid;
}

static void graphs_clear(Workspace& w) {
  for (auto g : w.graphs)
    if (g) cudaGraphExecDestroy(g);
  w.graphs.clear();
  w.graph_key = GraphKey();
}

int ws_prepare(qcd_ctx* c, Workspace& w, const qcd_solver_params& sp, cudaStream_t s) {
  const int nkv = sp.nkv;
  const int rprec = sp.outer_prec == P32 ? P32 : P64;
  for (Rec* f : {&w.b, &w.x, &w.r})
    if (!f->data) QCD_TRY(rec_alloc(*f, P64, 24, c->V));
  if (w.rprec != rprec) {  // the recursion vectors change precision: reallocate them
    graphs_clear(w);
    rec_free(w.rho);
    for (auto& r : w.phi) rec_free(r);
    for (auto& r : w.chi) rec_free(r);
    w.phi.clear();
    w.chi.clear();
    w.nkv = 0;
    w.rprec = rprec;
  }
  if (!w.rho.data) QCD_TRY(rec_alloc(w.rho, rprec, 24, c->V));
  if (!w.d_part) {
    if (cudaMalloc(&w.d_part, sizeof(double) * partials_for(c->V)) != cudaSuccess) {
      cudaGetLastError();
      w.d_part = nullptr;
      return QCD_ERR_NOMEM;
    }
  }
  if (nkv > w.nkv) {
    for (int k = w.nkv; k < nkv; ++k) {
      w.phi.emplace_back();
      w.chi.emplace_back();
      QCD_TRY(rec_alloc(w.phi.back(), rprec, 24, c->V));
      QCD_TRY(rec_alloc(w.chi.back(), rprec, 24, c->V));
    }
    cudaFree(w.d_a1);
    cudaFree(w.d_a2);
    cudaFree(w.d_cr);
    cudaFree(w.d_rn);
    cudaFree(w.d_gam);
    cudaFree(w.d_gs);
    if (w.h_pin) cudaFreeHost(w.h_pin);
    w.d_a1 = w.d_a2 = w.d_cr = w.d_rn = w.d_gam = w.d_gs = w.h_pin = nullptr;
    QCD_CUDA(cudaMalloc(&w.d_a1, sizeof(double) * 2 * nkv * nkv));
    QCD_CUDA(cudaMalloc(&w.d_a2, sizeof(double) * 2 * nkv * nkv));
    QCD_CUDA(cudaMalloc(&w.d_cr, sizeof(double) * 3 * nkv));
    QCD_CUDA(cudaMalloc(&w.d_rn, sizeof(double) * (nkv + 8)));
    QCD_CUDA(cudaMalloc(&w.d_gam, sizeof(double) * 2 * nkv));
    QCD_CUDA(cudaMalloc(&w.d_gs, sizeof(double) * 8 * nkv));
    QCD_CUDA(cudaMallocHost(&w.h_pin, sizeof(double) * (nkv + 8)));
    w.nkv = nkv;
  }
  QCD_TRY(ensure_gauge(c, P64, s));
  QCD_TRY(ensure_clover(c, P64, s));
  if (rprec != P64) {
    QCD_TRY(ensure_gauge(c, rprec, s));
    QCD_TRY(ensure_clover(c, rprec, s));
  }
  if (sp.precond == QCD_PRECOND_SAP) QCD_TRY(sap_prepare(c, w.sap, sp.sap_prec, s));
  return QCD_OK;
}

void ws_release(Workspace& w) {
  graphs_clear(w);
  dr_release(w);
  cg_release(w);
  if (w.stage) cudaFree(w.stage);
  w.stage = nullptr;
  w.stage_bytes = 0;
  rec_free(w.sap.rho);
  rec_free(w.sap.psi);
  if (w.sap.faces) cudaFree(w.sap.faces);
  w.sap.faces = nullptr;
  w.sap.prec = -1;
  for (Rec* f : {&w.b, &w.x, &w.r, &w.rho, &w.tmp64}) rec_free(*f);
  for (auto& r : w.phi) rec_free(r);
  for (auto& r : w.chi) rec_free(r);
  w.phi.clear();
  w.chi.clear();
  for (double** p : {&w.d_a1, &w.d_a2, &w.d_cr, &w.d_rn, &w.d_gam, &w.d_gs, &w.d_part}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  if (w.h_pin) cudaFreeHost(w.h_pin);
  w.h_pin = nullptr;
  w.nkv = 0;
  w.rprec = P64;
}

// classical Gram-Schmidt of chi_k against chi_0 .. chi_{k-1}, normalisation
// and residual update, in the recursion's precision R; the second pass runs
// (decided on the device) only if the first one cancelled more than half of
// the squared norm
template <typename R>
static int gram_schmidt(qcd_ctx* c, Workspace& w, const qcd_solver_params& sp, int k, cudaStream_t s) {
  NvtxRange nv("gram_schmidt");
  const R* chi_p[64];
  for (int j = 0; j < k; ++j) chi_p[j] = (const R*)w.chi[j].data;
  R* chik = (R*)w.chi[k].data;
  R* rho = (R*)w.rho.data;
  double* a1 = w.d_a1 + 2 * (size_t)k * sp.nkv;
  double* a2 = w.d_a2 + 2 * (size_t)k * sp.nkv;
  double* gs = w.d_gs + 8 * (size_t)k;
  QCD_TRY(blas_multidot<R>(c, w.d_part, chi_p, k, chik, a1, s, nullptr, gs));
  QCD_TRY(blas_axpy_norm_dot<R>(c, w.d_part, chi_p, k, a1, chik, rho, gs + 1, s));
  if (k > 0) {
    QCD_TRY(blas_multidot<R>(c, w.d_part, chi_p, k, chik, a2, s, gs));
    QCD_TRY(blas_axpy_norm_dot<R>(c, w.d_part, chi_p, k, a2, chik, rho, gs + 4, s, gs));
  }
  return blas_normalise_update<R>(c, w.d_part, chik, rho, gs, k > 0, w.d_cr + 3 * k, w.d_rn + k, s);
}

// enqueue FGCR iteration k of one problem; ends with a copy of |rho_{k+1}|^2
// to w.h_pin[k] (pinned host memory)
static int enqueue_iteration(Problem& p, const qcd_solver_params& sp, int k) {
  qcd_ctx* c = p.c;
  Workspace& w = *p.w;
  cudaStream_t s = p.s;
  if (sp.precond == QCD_PRECOND_SAP) {
    NvtxRange nv("sap");
    QCD_TRY(sap_apply(c, w.sap, w.rho, w.phi[k], sp.ncy, sp.nmr, sp.sap_prec, s));
  } else {
    QCD_CUDA(cudaMemcpyAsync(w.phi[k].data, w.rho.data, w.rho.bytes, cudaMemcpyDeviceToDevice, s));
  }
  {
    NvtxRange nv("outer_operator");
    QCD_TRY(dirac_apply(c, w.phi[k], w.chi[k], 0, s));
  }
  if (w.rprec == P32)
    QCD_TRY(gram_schmidt<float>(c, w, sp, k, s));
  else
    QCD_TRY(gram_schmidt<double>(c, w, sp, k, s));
  QCD_CUDA(cudaMemcpyAsync(w.h_pin + k, w.d_rn + k, sizeof(double), cudaMemcpyDeviceToHost, s));
  // the SAP staging time-out flag, so that a skipped block (whose garbage may
  // turn into a NaN) is reported as the time-out it is
  if (sp.precond == QCD_PRECOND_SAP)
    QCD_CUDA(cudaMemcpyAsync(w.h_pin + w.nkv + 4, c->d_scalars + 128, sizeof(double), cudaMemcpyDeviceToHost, s));
  return QCD_OK;
}

static GraphKey graph_key(const qcd_ctx* c, const qcd_solver_params& sp) {
  GraphKey k;
  k.gen = c->gen;
  k.nkv = sp.nkv;
  k.precond = sp.precond;
  k.ncy = sp.ncy;
  k.nmr = sp.nmr;
  k.sap_prec = sp.sap_prec;
  k.outer_prec = sp.outer_prec;
  return k;
}

// enqueue iteration k, from a captured graph when requested
static int launch_iteration(Problem& p, const qcd_solver_params& sp, int k, bool use_graphs) {
  if (!use_graphs) return enqueue_iteration(p, sp, k);
  Workspace& w = *p.w;
  const GraphKey key = graph_key(p.c, sp);
  if (w.graph_key != key) {
    graphs_clear(w);
    w.graphs.assign(sp.nkv, nullptr);
    w.graph_key = key;
  }
  if (!w.graphs[k]) {
    cudaGraph_t g = nullptr;
    QCD_CUDA(cudaStreamBeginCapture(p.s, cudaStreamCaptureModeThreadLocal));
    int st = enqueue_iteration(p, sp, k);
    cudaError_t e = cudaStreamEndCapture(p.s, &g);
    if (st != QCD_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&w.graphs[k], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      w.graphs[k] = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  QCD_CUDA(cudaGraphLaunch(w.graphs[k], p.s));
  return QCD_OK;
}

static int sync_all(std::vector<Problem>& probs) {
  for (auto& p : probs)
    if (p.active) QCD_CUDA(cudaStreamSynchronize(p.s));
  return QCD_OK;
}

int fgcr_batch(std::vector<Problem>& probs, const qcd_solver_params& sp, bool use_graphs) {
  NvtxRange nv("fgcr");
  if (sp.nkv < 1 || sp.nkv > 64 || !(sp.tol > 0) || sp.max_restarts < 1) return QCD_ERR_ARG;
  if (sp.precond != QCD_PRECOND_NONE && sp.precond != QCD_PRECOND_SAP) return QCD_ERR_ARG;
  if (sp.outer_prec != P64 && sp.outer_prec != P32) return QCD_ERR_ARG;
  if (sp.outer_prec == P32 && !(sp.inner_tol > 0 && sp.inner_tol < 1)) return QCD_ERR_ARG;
  if (sp.precond == QCD_PRECOND_SAP && (sp.ncy < 1 || sp.nmr < 0 || sp.sap_prec < P64 || sp.sap_prec > PB16))
    return QCD_ERR_ARG;
  const size_t bytes_of = sizeof(double);
  for (auto& p : probs) {
    memset(&p.info, 0, sizeof(p.info));
    p.active = true;
    p.status = QCD_OK;
    if (!p.c->clover_built) {
      p.status = QCD_ERR_STATE;
      p.active = false;
      continue;
    }
    int st = ws_prepare(p.c, *p.w, sp, p.s);
    // clear the SAP staging time-out flag of the context
    if (st == QCD_OK && cudaMemsetAsync(p.c->d_scalars + 128, 0, sizeof(double), p.s) != cudaSuccess)
      st = QCD_ERR_CUDA;
    if (st != QCD_OK) {
      p.status = st;
      p.active = false;
    }
  }
  // |b|^2 and |x0|^2; then r = b - D x0, or r = b without an operator
  // application when the initial guess is zero
  for (auto& p : probs) {
    if (!p.active) continue;
    Workspace& w = *p.w;
    int st = blas_norm2<double>(p.c, w.d_part, (const double*)p.b.data, w.d_rn + w.nkv, p.s);
    if (st == QCD_OK) st = blas_norm2<double>(p.c, w.d_part, (const double*)p.x.data, w.d_rn + w.nkv + 3, p.s);
    if (st == QCD_OK && cudaMemcpyAsync(w.h_pin + w.nkv, w.d_rn + w.nkv, 4 * bytes_of, cudaMemcpyDeviceToHost,
                                        p.s) != cudaSuccess)
      st = QCD_ERR_CUDA;
    if (st != QCD_OK) {
      p.status = st;
      p.active = false;
    }
  }
  QCD_TRY(sync_all(probs));
  for (auto& p : probs) {
    if (!p.active) continue;
    Workspace& w = *p.w;
    int st = QCD_OK;
    if (w.h_pin[w.nkv + 3] == 0.0) {
      if (cudaMemcpyAsync(w.r.data, p.b.data, w.r.bytes, cudaMemcpyDeviceToDevice, p.s) != cudaSuccess ||
          cudaMemcpyAsync(w.d_rn + w.nkv + 1, w.d_rn + w.nkv, bytes_of, cudaMemcpyDeviceToDevice, p.s) != cudaSuccess)
        st = QCD_ERR_CUDA;
    } else {
      st = residual64(p.c, w.d_part, p.b, p.x, w.r, w.d_rn + w.nkv + 1, p.s);
    }
    if (st == QCD_OK && cudaMemcpyAsync(w.h_pin + w.nkv + 1, w.d_rn + w.nkv + 1, bytes_of, cudaMemcpyDeviceToHost,
                                        p.s) != cudaSuccess)
      st = QCD_ERR_CUDA;
    if (st != QCD_OK) {
      p.status = st;
      p.active = false;
    }
  }
  QCD_TRY(sync_all(probs));
  for (auto& p : probs) {
    if (!p.active) continue;
    Workspace& w = *p.w;
    const double bn2 = w.h_pin[w.nkv], rn2 = w.h_pin[w.nkv + 1];
    if (!(bn2 == bn2) || std::isinf(bn2) || !(rn2 == rn2)) {
      p.status = QCD_NAN;
      p.active = false;
      continue;
    }
    if (bn2 == 0.0) {  // b = 0: x = 0
      if (cudaMemsetAsync(p.x.data, 0, (size_t)p.c->V * 24 * sizeof(double), p.s) != cudaSuccess)
        p.status = QCD_ERR_CUDA;
      p.active = false;
      continue;
    }
    p.bn = std::sqrt(bn2);
    p.rn = std::sqrt(rn2);
    p.info.true_residual = p.rn / p.bn;
    p.slow = 0;
    if (p.rn <= sp.tol * p.bn) p.active = false;
  }
  // restart cycles
  for (;;) {
    bool any = false;
    for (auto& p : probs) {
      if (p.active && p.info.restarts >= sp.max_restarts) {
        p.status = QCD_NOT_CONVERGED;
        p.active = false;
      }
      any |= p.active;
    }
    if (!any) break;
    // rho_0: the FP64 residual, or r / |r| in FP32; |r|^2 of the cycle start
    // is in d_rn[nkv + 1] (first cycle) or d_rn[nkv + 2] (after a restart)
    for (auto& p : probs) {
      if (!p.active) continue;
      Workspace& w = *p.w;
      p.kused = 0;
      p.cycle_done = false;
      const double* rn2 = w.d_rn + w.nkv + (p.info.restarts == 0 ? 1 : 2);
      int st = QCD_OK;
      if (w.rprec == P32)
        st = blas_demote_normalised(p.c, (const double*)w.r.data, rn2, (float*)w.rho.data, p.s);
      else if (cudaMemcpyAsync(w.rho.data, w.r.data, w.r.bytes, cudaMemcpyDeviceToDevice, p.s) != cudaSuccess)
        st = QCD_ERR_CUDA;
      if (st != QCD_OK) {
        p.status = st;
        p.active = false;
      }
    }
    for (int k = 0; k < sp.nkv; ++k) {
      bool launched = false;
      for (auto& p : probs) {
        if (!p.active || p.cycle_done) continue;
        int st = launch_iteration(p, sp, k, use_graphs);
        if (st != QCD_OK) {
          p.status = st;
          p.active = false;
          continue;
        }
        launched = true;
      }
      if (!launched) break;
      QCD_TRY(sync_all(probs));
      for (auto& p : probs) {
        if (!p.active || p.cycle_done) continue;
        const double rk2 = p.w->h_pin[k];
        ++p.info.iterations;
        p.kused = k + 1;
        int sap_err = 0;
        if (sp.precond == QCD_PRECOND_SAP) memcpy(&sap_err, p.w->h_pin + p.w->nkv + 4, sizeof(int));
        if (sap_err) {
          p.status = QCD_ERR_TIMEOUT;
          p.active = false;
          continue;
        }
        if (!(rk2 == rk2)) {
          p.status = QCD_NAN;
          p.active = false;
          continue;
        }
        // FP32 cycles work on r / |r|: stop at the target or after a drop by inner_tol
        const double thr = p.w->rprec == P32 ? std::max(sp.tol * p.bn / p.rn, sp.inner_tol) : sp.tol * p.bn;
        if (std::sqrt(rk2) <= thr) p.cycle_done = true;
      }
    }
    // x += sum gamma_k phi_k; r = b - D x (FP64)
    for (auto& p : probs) {
      if (!p.active || p.kused == 0) continue;
      Workspace& w = *p.w;
      int st = fgcr_backsub(w.d_a1, w.d_a2, w.d_cr, p.kused, sp.nkv, w.d_gam, p.s);
      if (st == QCD_OK && w.rprec == P32) {
        const float* phi_p[64];
        for (int j = 0; j < p.kused; ++j) phi_p[j] = (const float*)w.phi[j].data;
        const double* rn2 = w.d_rn + w.nkv + (p.info.restarts == 0 ? 1 : 2);
        st = blas_refine_update(p.c, phi_p, p.kused, w.d_gam, rn2, (double*)p.x.data, p.s);
      } else if (st == QCD_OK) {
        const double* phi_p[64];
        for (int j = 0; j < p.kused; ++j) phi_p[j] = (const double*)w.phi[j].data;
        st = blas_multi_axpy<double>(p.c, phi_p, p.kused, w.d_gam, (double*)p.x.data, p.s);
      }
      if (st == QCD_OK) st = residual64(p.c, w.d_part, p.b, p.x, w.r, w.d_rn + w.nkv + 2, p.s);
      if (st == QCD_OK && cudaMemcpyAsync(w.h_pin + w.nkv + 2, w.d_rn + w.nkv + 2, bytes_of, cudaMemcpyDeviceToHost,
                                          p.s) != cudaSuccess)
        st = QCD_ERR_CUDA;
      if (st == QCD_OK && cudaMemcpyAsync(w.h_pin + w.nkv + 3, (const double*)(p.c->d_scalars + 128), bytes_of,
                                          cudaMemcpyDeviceToHost, p.s) != cudaSuccess)
        st = QCD_ERR_CUDA;
      if (st != QCD_OK) {
        p.status = st;
        p.active = false;
      }
    }
    QCD_TRY(sync_all(probs));
    for (auto& p : probs) {
      if (!p.active) continue;
      Workspace& w = *p.w;
      ++p.info.restarts;
      int sap_err = 0;
      memcpy(&sap_err, w.h_pin + w.nkv + 3, sizeof(int));
      if (sap_err) {
        p.status = QCD_ERR_TIMEOUT;
        p.active = false;
        continue;
      }
      const double nrn = std::sqrt(w.h_pin[w.nkv + 2]);
      if (!(nrn == nrn)) {
        p.status = QCD_NAN;
        p.active = false;
        continue;
      }
      p.slow = nrn > 0.999 * p.rn ? p.slow + 1 : 0;
      p.rn = nrn;
      p.info.true_residual = nrn / p.bn;
      if (nrn <= sp.tol * p.bn) {
        p.active = false;
      } else if (p.slow >= 3) {
        p.status = QCD_STAGNATED;
        p.active = false;
      }
    }
  }
  int first = QCD_OK;
  for (auto& p : probs) {
    p.info.status = p.status;
    if (p.status != QCD_OK && first == QCD_OK) first = p.status;
  }
  return first;
}

// the solver sp.solver names on every problem, then (cg_fallback) CG from the
// iterate of a Krylov solve that stagnated or ran out of restarts (Sec. 4: CG
// for the most difficult cases)
int run_solver(std::vector<Problem>& probs, const qcd_solver_params& sp, bool use_graphs) {
  if (sp.solver < QCD_SOLVER_FGCR || sp.solver > QCD_SOLVER_CG_EO || sp.cg_fallback < 0 || sp.cg_fallback > 2)
    return QCD_ERR_ARG;
  const bool cg = sp.solver == QCD_SOLVER_CG || sp.solver == QCD_SOLVER_CG_EO;
  int st;
  if (cg)
    st = cg_batch(probs, sp, false);
  else if (sp.solver == QCD_SOLVER_FGMRES_DR)
    st = fgmres_dr_batch(probs, sp);
  else
    st = fgcr_batch(probs, sp, use_graphs);
  if (!cg && sp.cg_fallback && st != QCD_OK) {
    bool any = false;
    for (auto& p : probs) any |= (p.status == QCD_STAGNATED || p.status == QCD_NOT_CONVERGED);
    if (any) {
      cg_batch(probs, sp, true);
      st = QCD_OK;
      for (auto& p : probs)
        if (p.status != QCD_OK && st == QCD_OK) st = p.status;
    }
  }
  return st;
}

int solve_one(qcd_ctx* c, const Rec& b, const Rec& x, const qcd_solver_params& sp, qcd_solve_info* info,
              cudaStream_t s) {
  Workspace* w = ensure_ws(c);
  if (!w) return QCD_ERR_NOMEM;
  std::vector<Problem> probs(1);
  probs[0].c = c;
  probs[0].w = w;
  probs[0].s = s;
  probs[0].b = b;
  probs[0].x = x;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  int st = run_solver(probs, sp, false);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  probs[0].info.time_ms = ms;
  if (info) *info = probs[0].info;
  return st;
}

void workspace_free(qcd_ctx* c) {
  if (c->ws) {
    ws_release(*c->ws);
    delete c->ws;
    c->ws = nullptr;
  }
  for (auto* w : c->batch_ws) {
    ws_release(*w);
    delete w;
  }
  c->batch_ws.clear();
}

}  // namespace qcd
