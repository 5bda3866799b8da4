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
// sizes) are solved in lock step.  The right-hand sides of one lattice form a
// group that shares one workspace (their fields back to back): every kernel of
// an iteration runs over all of them at once -- the SAP sweep solves a tile of
// right-hand sides per CTA with the block's links and clover staged once, the
// operator loops over them per site, the Gram-Schmidt kernels take a grid
// dimension over them -- and a device mask switches off the right-hand sides
// whose cycle has ended.  Lattices of different sizes form one group each, on
// its own stream, so their kernels run concurrently.  One host
// synchronisation per iteration reads all the recursive residuals.  With
// use_graphs each group's iteration k is captured once as a CUDA graph and
// replayed (one launch instead of ~20).
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
  w.graph_warm.clear();
  w.graph_key = GraphKey();
}

Rec rhs_view(const Rec& f, int q, long long V) {
  Rec v = f;
  v.data = (char*)f.data + (size_t)q * V * chunks(f.prec, f.nreal) * 16;
  if (f.norm) v.norm = f.norm + (size_t)q * V;
  v.bytes = (size_t)V * chunks(f.prec, f.nreal) * 16 + (f.norm ? (size_t)V * sizeof(float) : 0);
  return v;
}

Batch batch_of(const Workspace& w, const int* mask) {
  Batch B;
  B.n = w.nr;
  B.ss = w.ss;
  B.ps = w.ps;
  B.mask = mask;
  B.k = nullptr;
  return B;
}

static void scalars_free(Workspace& w) {
  if (w.d_scal) cudaFree(w.d_scal);
  if (w.h_pin) cudaFreeHost(w.h_pin);
  if (w.d_mask) cudaFree(w.d_mask);
  if (w.h_mask) cudaFreeHost(w.h_mask);
  w.d_scal = w.d_a1 = w.d_a2 = w.d_cr = w.d_rn = w.d_gam = w.d_gs = w.h_pin = nullptr;
  w.d_mask = w.h_mask = w.d_k = w.h_k = nullptr;
  w.ss = 0;
}

static void fields_free(Workspace& w) {
  graphs_clear(w);
  for (Rec* f : {&w.b, &w.x, &w.r, &w.rho, &w.tmp64}) rec_free(*f);
  for (auto& r : w.phi) rec_free(r);
  for (auto& r : w.chi) rec_free(r);
  w.phi.clear();
  w.chi.clear();
  if (w.d_part) cudaFree(w.d_part);
  w.d_part = nullptr;
  w.ps = 0;
  scalars_free(w);
  w.nkv = 0;
}

int ws_prepare(qcd_ctx* c, Workspace& w, const qcd_solver_params& sp, cudaStream_t s, int nr) {
  const int nkv = sp.nkv;
  const int rprec = sp.outer_prec == P32 ? P32 : (sp.outer_prec == PDF ? PDF : P64);
  // phi_k, the preconditioner's output and the operator's input: with the
  // double-float recursion the SAP output is FP32-exact and is kept in FP32
  const int pprec = (rprec == PDF && sp.precond == QCD_PRECOND_SAP) ? P32 : rprec;
  if (nr < 1) return QCD_ERR_ARG;
  if (w.nr != nr) {  // the number of right-hand sides changes: reallocate every field
    fields_free(w);
    w.nr = nr;
  }
  const long long Vn = c->V * nr;
  for (Rec* f : {&w.b, &w.x, &w.r})
    if (!f->data) QCD_TRY(rec_alloc(*f, P64, 24, Vn));
  if (w.rprec != rprec || w.pprec != pprec) {  // the recursion vectors change precision: reallocate them
    graphs_clear(w);
    rec_free(w.rho);
    for (auto& r : w.phi) rec_free(r);
    for (auto& r : w.chi) rec_free(r);
    w.phi.clear();
    w.chi.clear();
    scalars_free(w);
    w.nkv = 0;
    w.rprec = rprec;
    w.pprec = pprec;
  }
  if (!w.rho.data) QCD_TRY(rec_alloc(w.rho, rprec, 24, Vn));
  if (!w.d_part) {
    w.ps = (long long)partials_for(c->V);
    if (cudaMalloc(&w.d_part, sizeof(double) * w.ps * nr) != cudaSuccess) {
      cudaGetLastError();
      w.d_part = nullptr;
      return QCD_ERR_NOMEM;
    }
  }
  if (nkv > w.nkv) {
    graphs_clear(w);
    for (int k = w.nkv; k < nkv; ++k) {
      w.phi.emplace_back();
      w.chi.emplace_back();
      QCD_TRY(rec_alloc(w.phi.back(), pprec, 24, Vn));
      QCD_TRY(rec_alloc(w.chi.back(), rprec, 24, Vn));
    }
    scalars_free(w);
    // one block of scalars per right-hand side: a1, a2 (2 nkv^2 each), cr (3 nkv),
    // rn (nkv + 8), gam (2 nkv), gs (8 nkv)
    const long long ss = 4LL * nkv * nkv + 3 * nkv + (nkv + 8) + 2 * nkv + 8 * nkv;
    QCD_CUDA(cudaMalloc(&w.d_scal, sizeof(double) * ss * nr));
    QCD_CUDA(cudaMemset(w.d_scal, 0, sizeof(double) * ss * nr));
    w.ss = ss;
    w.d_a1 = w.d_scal;
    w.d_a2 = w.d_a1 + 2LL * nkv * nkv;
    w.d_cr = w.d_a2 + 2LL * nkv * nkv;
    w.d_rn = w.d_cr + 3 * nkv;
    w.d_gam = w.d_rn + nkv + 8;
    w.d_gs = w.d_gam + 2 * nkv;
    QCD_CUDA(cudaMallocHost(&w.h_pin, sizeof(double) * (nkv + 8) * nr));
    QCD_CUDA(cudaMalloc(&w.d_mask, sizeof(int) * 2 * nr));
    QCD_CUDA(cudaMallocHost(&w.h_mask, sizeof(int) * 2 * nr));
    w.d_k = w.d_mask + nr;
    w.h_k = w.h_mask + nr;
    w.nkv = nkv;
  }
  QCD_TRY(ensure_gauge(c, P64, s));
  QCD_TRY(ensure_clover(c, P64, s));
  if (rprec != P64) {  // the outer operator's links and clover in the recursion's precision
    QCD_TRY(ensure_gauge(c, rprec, s));
    QCD_TRY(ensure_clover(c, rprec, s));
  }
  if (sp.precond == QCD_PRECOND_SAP) QCD_TRY(sap_prepare(c, w.sap, sp.sap_prec, s, nr));
  return QCD_OK;
}

void ws_release(Workspace& w) {
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
  w.sap.nr = 0;
  fields_free(w);
  w.nr = 1;
  w.rprec = P64;
}

// classical Gram-Schmidt of chi_k against chi_0 .. chi_{k-1}, normalisation
// and residual update, in the recursion's precision R, for every right-hand
// side of B; the second pass runs (decided on the device, per right-hand
// side) only if the first one cancelled more than half of the squared norm
template <typename R>
static int gram_schmidt(qcd_ctx* c, Workspace& w, const qcd_solver_params& sp, int k, cudaStream_t s,
                        const Batch& B) {
  NvtxRange nv("gram_schmidt");
  const R* chi_p[64];
  for (int j = 0; j < k; ++j) chi_p[j] = (const R*)w.chi[j].data;
  R* chik = (R*)w.chi[k].data;
  R* rho = (R*)w.rho.data;
  double* a1 = w.d_a1 + 2 * (size_t)k * sp.nkv;
  double* a2 = w.d_a2 + 2 * (size_t)k * sp.nkv;
  double* gs = w.d_gs + 8 * (size_t)k;
  QCD_TRY(blas_multidot<R>(c, w.d_part, chi_p, k, chik, a1, s, nullptr, gs, B));
  QCD_TRY(blas_axpy_norm_dot<R>(c, w.d_part, chi_p, k, a1, chik, rho, gs + 1, s, nullptr, B));
  if (k > 0) {
    QCD_TRY(blas_multidot<R>(c, w.d_part, chi_p, k, chik, a2, s, gs, nullptr, B));
    QCD_TRY(blas_axpy_norm_dot<R>(c, w.d_part, chi_p, k, a2, chik, rho, gs + 4, s, gs, B));
  }
  return blas_normalise_update<R>(c, w.d_part, chik, rho, gs, k > 0, w.d_cr + 3 * k, w.d_rn + k, s, B);
}

// the same on the double-float fields of the df64 recursion
static int gram_schmidt_df(qcd_ctx* c, Workspace& w, const qcd_solver_params& sp, int k, cudaStream_t s,
                           const Batch& B) {
  NvtxRange nv("gram_schmidt");
  const float4* chi_p[64];
  for (int j = 0; j < k; ++j) chi_p[j] = (const float4*)w.chi[j].data;
  float4* chik = (float4*)w.chi[k].data;
  float4* rho = (float4*)w.rho.data;
  double* a1 = w.d_a1 + 2 * (size_t)k * sp.nkv;
  double* a2 = w.d_a2 + 2 * (size_t)k * sp.nkv;
  double* gs = w.d_gs + 8 * (size_t)k;
  QCD_TRY(blas_df_multidot(c, w.d_part, chi_p, k, chik, a1, s, nullptr, gs, B));
  QCD_TRY(blas_df_axpy_norm_dot(c, w.d_part, chi_p, k, a1, chik, rho, gs + 1, s, nullptr, B));
  if (k > 0) {
    QCD_TRY(blas_df_multidot(c, w.d_part, chi_p, k, chik, a2, s, gs, nullptr, B));
    QCD_TRY(blas_df_axpy_norm_dot(c, w.d_part, chi_p, k, a2, chik, rho, gs + 4, s, gs, B));
  }
  return blas_df_normalise_update(c, w.d_part, chik, rho, gs, k > 0, w.d_cr + 3 * k, w.d_rn + k, s, B);
}

// copy scalar j of every right-hand side's rn block to column j of the pinned mirror
static int read_rn(const Workspace& w, int j, cudaStream_t s) {
  const size_t dsz = sizeof(double);
  if (w.nr == 1) {
    QCD_CUDA(cudaMemcpyAsync(w.h_pin + j, w.d_rn + j, dsz, cudaMemcpyDeviceToHost, s));
  } else {
    QCD_CUDA(cudaMemcpy2DAsync(w.h_pin + j, dsz * (w.nkv + 8), w.d_rn + j, dsz * w.ss, dsz, w.nr,
                               cudaMemcpyDeviceToHost, s));
  }
  return QCD_OK;
}

static const int* group_mask(const Group& G) { return G.nr() > 1 ? G.w->d_mask : nullptr; }

// enqueue FGCR iteration k of one group; ends with a copy of every right-hand
// side's |rho_{k+1}|^2 to row q, column k of w.h_pin (pinned host memory)
static int enqueue_iteration(Group& G, const qcd_solver_params& sp, int k) {
  qcd_ctx* c = G.c;
  Workspace& w = *G.w;
  cudaStream_t s = G.s;
  const Batch B = batch_of(w, group_mask(G));
  if (sp.precond == QCD_PRECOND_SAP) {
    NvtxRange nv("sap");
    QCD_TRY(sap_apply(c, w.sap, w.rho, w.phi[k], sp.ncy, sp.nmr, sp.sap_prec, s, B, G.rt));
  } else {
    QCD_CUDA(cudaMemcpyAsync(w.phi[k].data, w.rho.data, w.rho.bytes, cudaMemcpyDeviceToDevice, s));
  }
  {
    NvtxRange nv("outer_operator");
    QCD_TRY(dirac_apply(c, w.phi[k], w.chi[k], 0, s, w.nr, B.mask));
  }
  if (w.rprec == P32)
    QCD_TRY(gram_schmidt<float>(c, w, sp, k, s, B));
  else if (w.rprec == PDF)
    QCD_TRY(gram_schmidt_df(c, w, sp, k, s, B));
  else
    QCD_TRY(gram_schmidt<double>(c, w, sp, k, s, B));
  QCD_TRY(read_rn(w, k, s));
  // the SAP staging time-out flag, so that a skipped block (whose garbage may
  // turn into a NaN) is reported as the time-out it is
  if (sp.precond == QCD_PRECOND_SAP)
    QCD_CUDA(cudaMemcpyAsync(&w.h_pin[w.nkv + 4], c->d_scalars + 128, sizeof(double), cudaMemcpyDeviceToHost, s));
  return QCD_OK;
}

static GraphKey graph_key(const Group& G, const qcd_solver_params& sp) {
  GraphKey k;
  k.gen = G.c->gen;
  k.nkv = sp.nkv;
  k.precond = sp.precond;
  k.ncy = sp.ncy;
  k.nmr = sp.nmr;
  k.sap_prec = sp.sap_prec;
  k.outer_prec = sp.outer_prec;
  k.nr = G.nr();
  k.rt = G.rt;
  return k;
}

// enqueue iteration k, from a captured graph when requested.  The first time
// an iteration index runs under a key it runs eagerly: kernels are loaded on
// their first launch (lazy module loading), which a stream capture does not
// permit, so only iterations whose kernels have all run are captured.
static int launch_iteration(Group& G, const qcd_solver_params& sp, int k, bool use_graphs) {
  if (!use_graphs) return enqueue_iteration(G, sp, k);
  Workspace& w = *G.w;
  const GraphKey key = graph_key(G, sp);
  if (w.graph_key != key) {
    graphs_clear(w);
    w.graphs.assign(sp.nkv, nullptr);
    w.graph_warm.assign(sp.nkv, 0);
    w.graph_key = key;
  }
  if (!w.graph_warm[k]) {
    w.graph_warm[k] = 1;
    return enqueue_iteration(G, sp, k);
  }
  if (!w.graphs[k]) {
    cudaGraph_t g = nullptr;
    QCD_CUDA(cudaStreamBeginCapture(G.s, cudaStreamCaptureModeThreadLocal));
    int st = enqueue_iteration(G, sp, k);
    cudaError_t e = cudaStreamEndCapture(G.s, &g);
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
  QCD_CUDA(cudaGraphLaunch(w.graphs[k], G.s));
  return QCD_OK;
}

// upload the group's mask: right-hand side q takes part iff on(q)
template <typename F>
static int upload_mask(Group& G, F on) {
  if (G.nr() == 1) return QCD_OK;
  Workspace& w = *G.w;
  for (int q = 0; q < G.nr(); ++q) w.h_mask[q] = on(*G.rhs[q]) ? 1 : 0;
  QCD_CUDA(cudaMemcpyAsync(w.d_mask, w.h_mask, sizeof(int) * G.nr(), cudaMemcpyHostToDevice, G.s));
  return QCD_OK;
}

static int sync_groups(std::vector<Group>& groups) {
  for (auto& G : groups) {
    bool any = false;
    for (auto* p : G.rhs) any |= p->active;
    if (any) QCD_CUDA(cudaStreamSynchronize(G.s));
  }
  return QCD_OK;
}

static bool group_active(const Group& G) {
  for (auto* p : G.rhs)
    if (p->active) return true;
  return false;
}

static void group_fail(Group& G, int st) {
  for (auto* p : G.rhs)
    if (p->active) {
      p->status = st;
      p->active = false;
    }
}

int fgcr_groups(std::vector<Group>& groups, const qcd_solver_params& sp, bool use_graphs) {
  NvtxRange nv("fgcr");
  if (sp.nkv < 1 || sp.nkv > 64 || !(sp.tol > 0) || sp.max_restarts < 1) return QCD_ERR_ARG;
  if (sp.precond != QCD_PRECOND_NONE && sp.precond != QCD_PRECOND_SAP) return QCD_ERR_ARG;
  if (sp.outer_prec != P64 && sp.outer_prec != P32 && sp.outer_prec != PDF) return QCD_ERR_ARG;
  if (sp.outer_prec == P32 && !(sp.inner_tol > 0 && sp.inner_tol < 1)) return QCD_ERR_ARG;
  if (sp.residual_prec != P64 && sp.residual_prec != PDF) return QCD_ERR_ARG;
  // restart residuals of the double-float recursion from a double-float D x unless FP64 is asked for
  const bool res_df = sp.outer_prec == PDF && sp.residual_prec == PDF;
  if (sp.precond == QCD_PRECOND_SAP && (sp.ncy < 1 || sp.nmr < 0 || sp.sap_prec < P64 || sp.sap_prec > PB16))
    return QCD_ERR_ARG;
  const size_t dsz = sizeof(double);
  for (auto& G : groups) {
    for (auto* p : G.rhs) {
      memset(&p->info, 0, sizeof(p->info));
      p->active = true;
      p->status = QCD_OK;
    }
    int st = G.c->clover_built ? QCD_OK : QCD_ERR_STATE;
    if (st == QCD_OK && G.w->nr != G.nr()) st = QCD_ERR_ARG;  // the caller prepared the workspace
    if (st == QCD_OK) st = ws_prepare(G.c, *G.w, sp, G.s, G.nr());
    // clear the SAP staging time-out flag of the context
    if (st == QCD_OK && cudaMemsetAsync(G.c->d_scalars + 128, 0, dsz, G.s) != cudaSuccess) st = QCD_ERR_CUDA;
    if (st != QCD_OK) group_fail(G, st);
  }
  // |b|^2 and |x0|^2 of every right-hand side; then r = b - D x0, or r = b
  // without an operator application when every initial guess is zero
  for (auto& G : groups) {
    if (!group_active(G)) continue;
    Workspace& w = *G.w;
    const Batch B = batch_of(w, nullptr);
    int st = blas_norm2<double>(G.c, w.d_part, (const double*)w.b.data, w.d_rn + w.nkv, G.s, B);
    if (st == QCD_OK) st = read_rn(w, w.nkv, G.s);
    if (sp.zero_guess) {  // the caller stated x = 0 (and the API cleared it): no norm to take
      for (int q = 0; q < G.nr(); ++q) w.h_pin[q * (w.nkv + 8) + w.nkv + 3] = 0.0;
    } else {
      if (st == QCD_OK) st = blas_norm2<double>(G.c, w.d_part, (const double*)w.x.data, w.d_rn + w.nkv + 3, G.s, B);
      if (st == QCD_OK) st = read_rn(w, w.nkv + 3, G.s);
    }
    if (st != QCD_OK) group_fail(G, st);
  }
  QCD_TRY(sync_groups(groups));
  for (auto& G : groups) {
    if (!group_active(G)) continue;
    Workspace& w = *G.w;
    const int hp = w.nkv + 8;
    bool zero = true;
    for (int q = 0; q < G.nr(); ++q) zero &= w.h_pin[q * hp + w.nkv + 3] == 0.0;
    int st = QCD_OK;
    if (zero) {  // r = b and |r|^2 = |b|^2 (on the device too: the FP32 recursion reads it there)
      if (cudaMemcpyAsync(w.r.data, w.b.data, w.r.bytes, cudaMemcpyDeviceToDevice, G.s) != cudaSuccess ||
          cudaMemcpy2DAsync(w.d_rn + w.nkv + 1, sizeof(double) * w.ss, w.d_rn + w.nkv, sizeof(double) * w.ss,
                            sizeof(double), G.nr(), cudaMemcpyDeviceToDevice, G.s) != cudaSuccess)
        st = QCD_ERR_CUDA;
      for (int q = 0; q < G.nr() && st == QCD_OK; ++q) w.h_pin[q * hp + w.nkv + 1] = w.h_pin[q * hp + w.nkv];
    } else {
      st = res_df ? residual_df(G.c, w.d_part, w.b, w.x, w.r, w.chi[0], w.d_rn + w.nkv + 1, G.s, batch_of(w, nullptr))
                  : residual64(G.c, w.d_part, w.b, w.x, w.r, w.d_rn + w.nkv + 1, G.s, batch_of(w, nullptr));
      if (st == QCD_OK) st = read_rn(w, w.nkv + 1, G.s);
    }
    if (st != QCD_OK) group_fail(G, st);
  }
  QCD_TRY(sync_groups(groups));
  for (auto& G : groups) {
    if (!group_active(G)) continue;
    Workspace& w = *G.w;
    const int hp = w.nkv + 8;
    for (int q = 0; q < G.nr(); ++q) {
      Problem& p = *G.rhs[q];
      const double bn2 = w.h_pin[q * hp + w.nkv], rn2 = w.h_pin[q * hp + w.nkv + 1];
      if (!(bn2 == bn2) || std::isinf(bn2) || !(rn2 == rn2)) {
        p.status = QCD_NAN;
        p.active = false;
        continue;
      }
      if (bn2 == 0.0) {  // b = 0: x = 0
        if (cudaMemsetAsync(p.x.data, 0, (size_t)G.c->V * 24 * sizeof(double), G.s) != cudaSuccess)
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
  }
  // its |r|^2 at the start of a cycle: rn[nkv + 1] (first cycle) or rn[nkv + 2]
  // (after a restart); the restart counts of the active right-hand sides agree
  int cycles = 0;
  for (;;) {
    bool any = false;
    for (auto& G : groups)
      for (auto* p : G.rhs) {
        if (p->active && p->info.restarts >= sp.max_restarts) {
          p->status = QCD_NOT_CONVERGED;
          p->active = false;
        }
        any |= p->active;
      }
    if (!any) break;
    // rho_0: the FP64 residual, or r / |r| in FP32
    for (auto& G : groups) {
      if (!group_active(G)) continue;
      Workspace& w = *G.w;
      for (auto* p : G.rhs) {
        p->kused = 0;
        p->cycle_done = !p->active;
      }
      const double* rn2 = w.d_rn + w.nkv + (cycles == 0 ? 1 : 2);
      int st = QCD_OK;
      if (w.rprec == P32)
        st = blas_demote_normalised(G.c, (const double*)w.r.data, rn2, (float*)w.rho.data, G.s,
                                    batch_of(w, nullptr));
      else if (w.rprec == PDF)
        st = blas_df_split(G.c, (const double*)w.r.data, (float*)w.rho.data, G.s, batch_of(w, nullptr));
      else if (cudaMemcpyAsync(w.rho.data, w.r.data, w.r.bytes, cudaMemcpyDeviceToDevice, G.s) != cudaSuccess)
        st = QCD_ERR_CUDA;
      if (st != QCD_OK) group_fail(G, st);
    }
    for (int k = 0; k < sp.nkv; ++k) {
      bool launched = false;
      for (auto& G : groups) {
        bool run = false;
        for (auto* p : G.rhs) run |= (p->active && !p->cycle_done);
        if (!run) continue;
        int st = upload_mask(G, [](const Problem& p) { return p.active && !p.cycle_done; });
        if (st == QCD_OK) st = launch_iteration(G, sp, k, use_graphs);
        if (st != QCD_OK) {
          group_fail(G, st);
          continue;
        }
        launched = true;
      }
      if (!launched) break;
      QCD_TRY(sync_groups(groups));
      for (auto& G : groups) {
        Workspace& w = *G.w;
        const int hp = w.nkv + 8;
        int sap_err = 0;
        if (sp.precond == QCD_PRECOND_SAP) memcpy(&sap_err, &w.h_pin[w.nkv + 4], sizeof(int));
        for (int q = 0; q < G.nr(); ++q) {
          Problem& p = *G.rhs[q];
          if (!p.active || p.cycle_done) continue;
          const double rk2 = w.h_pin[q * hp + k];
          ++p.info.iterations;
          p.kused = k + 1;
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
          const double thr = w.rprec == P32 ? std::max(sp.tol * p.bn / p.rn, sp.inner_tol) : sp.tol * p.bn;
          if (std::sqrt(rk2) <= thr) p.cycle_done = true;
        }
      }
    }
    // x += sum gamma_k phi_k; r = b - D x (FP64), for the right-hand sides
    // that iterated in this cycle
    for (auto& G : groups) {
      Workspace& w = *G.w;
      int kmax = 0;
      for (auto* p : G.rhs)
        if (p->active) kmax = std::max(kmax, p->kused);
      if (kmax == 0) continue;
      int st = upload_mask(G, [](const Problem& p) { return p.active && p.kused > 0; });
      Batch B = batch_of(w, group_mask(G));
      if (st == QCD_OK && G.nr() > 1) {
        for (int q = 0; q < G.nr(); ++q) w.h_k[q] = G.rhs[q]->kused;
        if (cudaMemcpyAsync(w.d_k, w.h_k, sizeof(int) * G.nr(), cudaMemcpyHostToDevice, G.s) != cudaSuccess)
          st = QCD_ERR_CUDA;
        B.k = w.d_k;
      }
      if (st == QCD_OK) st = fgcr_backsub(w.d_a1, w.d_a2, w.d_cr, kmax, sp.nkv, w.d_gam, G.s, B);
      // x changes below: a delivery of the previous x must have read it first
      for (auto* p : G.rhs)
        if (p->dlv_event && cudaStreamWaitEvent(G.s, p->dlv_event, 0) != cudaSuccess) st = QCD_ERR_CUDA;
      for (auto* p : G.rhs) p->delivered = false;
      if (st == QCD_OK && w.rprec == P32) {
        const float* phi_p[64];
        for (int j = 0; j < kmax; ++j) phi_p[j] = (const float*)w.phi[j].data;
        const double* rn2 = w.d_rn + w.nkv + (cycles == 0 ? 1 : 2);
        st = blas_refine_update(G.c, phi_p, kmax, w.d_gam, rn2, (double*)w.x.data, G.s, B);
      } else if (st == QCD_OK && w.rprec == PDF) {
        const float4* phi_p[64];
        for (int j = 0; j < kmax; ++j) phi_p[j] = (const float4*)w.phi[j].data;
        // with the FP32 phi the update also leaves the split of x for the residual in chi_0
        st = w.pprec == P32 ? blas_df_update32(G.c, phi_p, kmax, w.d_gam, (double*)w.x.data, G.s, B,
                                               res_df ? (float*)w.chi[0].data : nullptr)
                            : blas_df_update(G.c, phi_p, kmax, w.d_gam, (double*)w.x.data, G.s, B);
      } else if (st == QCD_OK) {
        const double* phi_p[64];
        for (int j = 0; j < kmax; ++j) phi_p[j] = (const double*)w.phi[j].data;
        st = blas_multi_axpy<double>(G.c, phi_p, kmax, w.d_gam, (double*)w.x.data, G.s, B);
      }
      // the updated x to the caller while the residual decides whether it is final
      if (st == QCD_OK && G.nr() == 1 && G.rhs[0]->dlv_lex) st = deliver_solution(*G.rhs[0], G.s);
      if (st == QCD_OK)  // (chi_0 is free: this cycle's Gram-Schmidt was its last use)
        st = res_df ? residual_df(G.c, w.d_part, w.b, w.x, w.r, w.chi[0], w.d_rn + w.nkv + 2, G.s, B,
                                  w.rprec == PDF && w.pprec == P32)
                    : residual64(G.c, w.d_part, w.b, w.x, w.r, w.d_rn + w.nkv + 2, G.s, B);
      if (st == QCD_OK) st = read_rn(w, w.nkv + 2, G.s);
      if (st == QCD_OK && cudaMemcpyAsync(&w.h_pin[w.nkv + 3], (const double*)(G.c->d_scalars + 128), dsz,
                                          cudaMemcpyDeviceToHost, G.s) != cudaSuccess)
        st = QCD_ERR_CUDA;
      if (st != QCD_OK) group_fail(G, st);
    }
    QCD_TRY(sync_groups(groups));
    ++cycles;
    for (auto& G : groups) {
      Workspace& w = *G.w;
      const int hp = w.nkv + 8;
      int sap_err = 0;
      memcpy(&sap_err, &w.h_pin[w.nkv + 3], sizeof(int));
      for (int q = 0; q < G.nr(); ++q) {
        Problem& p = *G.rhs[q];
        if (!p.active) continue;
        ++p.info.restarts;
        if (sap_err) {
          p.status = QCD_ERR_TIMEOUT;
          p.active = false;
          continue;
        }
        if (p.kused == 0) continue;
        const double nrn = std::sqrt(w.h_pin[q * hp + w.nkv + 2]);
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
  }
  int first = QCD_OK;
  for (auto& G : groups)
    for (auto* p : G.rhs) {
      p->info.status = p->status;
      if (p->status != QCD_OK && first == QCD_OK) first = p->status;
    }
  return first;
}

int fgcr_batch(std::vector<Problem>& probs, const qcd_solver_params& sp, bool use_graphs) {
  // one group per problem; the problems' b and x are the workspaces' own fields
  std::vector<Group> groups(probs.size());
  for (size_t i = 0; i < probs.size(); ++i) {
    Problem& p = probs[i];
    Group& G = groups[i];
    G.c = p.c;
    G.w = p.w;
    G.s = p.s;
    G.rt = 1;
    G.rhs.push_back(&p);
    if (p.w->nr != 1 || p.b.data != p.w->b.data || p.x.data != p.w->x.data) {
      // the problem's fields must be the workspace's: copy them in
      int st = ws_prepare(p.c, *p.w, sp, p.s, 1);
      if (st != QCD_OK) return st;
      if (p.b.data != p.w->b.data)
        QCD_CUDA(cudaMemcpyAsync(p.w->b.data, p.b.data, p.w->b.bytes, cudaMemcpyDeviceToDevice, p.s));
      if (p.x.data != p.w->x.data)
        QCD_CUDA(cudaMemcpyAsync(p.w->x.data, p.x.data, p.w->x.bytes, cudaMemcpyDeviceToDevice, p.s));
    }
  }
  std::vector<Rec> xs(probs.size());
  for (size_t i = 0; i < probs.size(); ++i) xs[i] = probs[i].x;
  for (size_t i = 0; i < probs.size(); ++i) {
    probs[i].b = probs[i].w->b;
    probs[i].x = probs[i].w->x;
  }
  const int st = fgcr_groups(groups, sp, use_graphs);
  for (size_t i = 0; i < probs.size(); ++i) {
    Problem& p = probs[i];
    if (xs[i].data != p.x.data) {  // hand the solution back to the caller's field
      if (cudaMemcpyAsync(xs[i].data, p.x.data, p.x.bytes, cudaMemcpyDeviceToDevice, p.s) != cudaSuccess &&
          p.status == QCD_OK)
        p.status = p.info.status = QCD_ERR_CUDA;
      p.x = xs[i];
    }
  }
  return st;
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
      for (auto& p : probs) {  // the fallback goes on from x: after any delivery of it has read it
        p.delivered = false;
        if (p.dlv_event) cudaStreamWaitEvent(p.s, p.dlv_event, 0);
      }
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
  for (Workspace** w : {&c->ws, &c->tile_ws})
    if (*w) {
      ws_release(**w);
      delete *w;
      *w = nullptr;
    }
  for (auto* w : c->batch_ws) {
    ws_release(*w);
    delete w;
  }
  c->batch_ws.clear();
}

}  // namespace qcd
