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
// the device, x += sum_k gamma_k phi_k, and r = b - D x is recomputed in FP64
// ("only when the FGCR recursion is restarted, the residue is computed in
// full double precision", Sec. 4).
#include <cmath>
#include <cstring>

#include "internal.h"

namespace qcd {

static int ws_reserve(qcd_ctx* c, Workspace& w, int nkv) {
  for (Rec* f : {&w.b, &w.x, &w.r, &w.rho})
    if (!f->data) QCD_TRY(rec_alloc(*f, P64, 24, c->V));
  if (nkv > w.nkv) {
    for (int k = w.nkv; k < nkv; ++k) {
      w.phi.emplace_back();
      w.chi.emplace_back();
      QCD_TRY(rec_alloc(w.phi.back(), P64, 24, c->V));
      QCD_TRY(rec_alloc(w.chi.back(), P64, 24, c->V));
    }
    cudaFree(w.d_a1);
    cudaFree(w.d_a2);
    cudaFree(w.d_cr);
    cudaFree(w.d_rn);
    cudaFree(w.d_gam);
    cudaFree(w.d_gs);
    cudaFreeHost(w.h_pin);
    QCD_CUDA(cudaMalloc(&w.d_a1, sizeof(double) * 2 * nkv * nkv));
    QCD_CUDA(cudaMalloc(&w.d_a2, sizeof(double) * 2 * nkv * nkv));
    QCD_CUDA(cudaMalloc(&w.d_cr, sizeof(double) * 3 * nkv));
    QCD_CUDA(cudaMalloc(&w.d_rn, sizeof(double) * (nkv + 8)));
    QCD_CUDA(cudaMalloc(&w.d_gam, sizeof(double) * 2 * nkv));
    QCD_CUDA(cudaMalloc(&w.d_gs, sizeof(double) * 8 * nkv));
    QCD_CUDA(cudaMallocHost(&w.h_pin, sizeof(double) * (nkv + 8)));
    w.nkv = nkv;
  }
  return QCD_OK;
}

// read one device double back (synchronises the stream)
static int read_scalar(Workspace& w, const double* d, double* h, cudaStream_t s) {
  QCD_CUDA(cudaMemcpyAsync(w.h_pin, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  *h = w.h_pin[0];
  return QCD_OK;
}

// chi = D phi in the requested outer precision (FP64 default)
static int outer_apply(qcd_ctx* c, Workspace& w, const Rec& phi, const Rec& chi, int prec, cudaStream_t s) {
  if (prec == P64) return dirac_apply(c, phi, chi, 0, s);
  if (w.lo_in.prec != prec) {
    rec_free(w.lo_in);
    rec_free(w.lo_out);
    QCD_TRY(rec_alloc(w.lo_in, prec, 24, c->V));
    QCD_TRY(rec_alloc(w.lo_out, prec, 24, c->V));
  }
  QCD_TRY(convert_rec(c, phi, w.lo_in, s));
  QCD_TRY(dirac_apply(c, w.lo_in, w.lo_out, 0, s));
  return convert_rec(c, w.lo_out, chi, s);
}

int solve_one(qcd_ctx* c, const Rec& b, const Rec& x, const qcd_solver_params& sp, qcd_solve_info* info,
              cudaStream_t s) {
  qcd_solve_info inf;
  memset(&inf, 0, sizeof(inf));
  auto finish = [&](int st) {
    inf.status = st;
    if (info) *info = inf;
    return st;
  };
  if (!c->clover_built) return finish(QCD_ERR_STATE);
  if (sp.nkv < 1 || sp.nkv > 64 || sp.tol <= 0 || sp.max_restarts < 1) return finish(QCD_ERR_ARG);
  if (sp.precond != QCD_PRECOND_NONE && sp.precond != QCD_PRECOND_SAP) return finish(QCD_ERR_ARG);
  if (sp.outer_prec != P64 && sp.outer_prec != P32) return finish(QCD_ERR_ARG);
  Workspace* wp = ensure_ws(c);
  if (!wp) return finish(QCD_ERR_NOMEM);
  Workspace& w = *wp;
  int st = ws_reserve(c, w, sp.nkv);
  if (st) return finish(st);

  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);

  auto run = [&]() -> int {
    const size_t bytes = (size_t)c->V * 24 * sizeof(double);
    double bn2 = 0, rn2 = 0;
    QCD_TRY(blas_norm2(c, (const double*)b.data, w.d_rn, s));
    QCD_TRY(read_scalar(w, w.d_rn, &bn2, s));
    if (!(bn2 == bn2) || std::isinf(bn2)) return QCD_NAN;
    if (bn2 == 0.0) {
      QCD_CUDA(cudaMemsetAsync(x.data, 0, bytes, s));
      inf.true_residual = 0;
      return QCD_OK;
    }
    const double bn = std::sqrt(bn2);
    QCD_TRY(residual64(c, b, x, w.r, w.d_rn, s));
    QCD_TRY(read_scalar(w, w.d_rn, &rn2, s));
    double rn = std::sqrt(rn2);
    inf.true_residual = rn / bn;
    if (!(rn == rn)) return QCD_NAN;
    int slow_cycles = 0;
    std::vector<const double*> chi_p(sp.nkv), phi_p(sp.nkv);
    for (int k = 0; k < sp.nkv; ++k) {
      chi_p[k] = (const double*)w.chi[k].data;
      phi_p[k] = (const double*)w.phi[k].data;
    }
    while (rn > sp.tol * bn && inf.restarts < sp.max_restarts) {
      QCD_CUDA(cudaMemcpyAsync(w.rho.data, w.r.data, bytes, cudaMemcpyDeviceToDevice, s));
      int kused = 0;
      for (int k = 0; k < sp.nkv; ++k) {
        if (sp.precond == QCD_PRECOND_SAP) {
          QCD_TRY(sap_apply(c, w.rho, w.phi[k], sp.ncy, sp.nmr, sp.sap_prec, s));
        } else {
          QCD_CUDA(cudaMemcpyAsync(w.phi[k].data, w.rho.data, bytes, cudaMemcpyDeviceToDevice, s));
        }
        QCD_TRY(outer_apply(c, w, w.phi[k], w.chi[k], sp.outer_prec, s));
        double* chik = (double*)w.chi[k].data;
        double* a1 = w.d_a1 + 2 * (size_t)k * sp.nkv;
        double* a2 = w.d_a2 + 2 * (size_t)k * sp.nkv;
        // classical Gram-Schmidt; the second pass runs (decided on the device)
        // only if the first one cancelled more than half of the squared norm
        double* gs = w.d_gs + 8 * (size_t)k;
        const double* rho_p = (const double*)w.rho.data;
        QCD_TRY(blas_multidot(c, chi_p.data(), k, chik, a1, s, nullptr, gs));
        QCD_TRY(blas_axpy_norm_dot(c, chi_p.data(), k, a1, chik, rho_p, gs + 1, s));
        if (k > 0) {
          QCD_TRY(blas_multidot(c, chi_p.data(), k, chik, a2, s, gs));
          QCD_TRY(blas_axpy_norm_dot(c, chi_p.data(), k, a2, chik, rho_p, gs + 4, s, gs));
        }
        QCD_TRY(blas_normalise_update(c, chik, (double*)w.rho.data, gs, k > 0, w.d_cr + 3 * k, w.d_rn + k, s));
        double rk2 = 0;
        QCD_TRY(read_scalar(w, w.d_rn + k, &rk2, s));
        ++inf.iterations;
        kused = k + 1;
        if (!(rk2 == rk2)) return QCD_NAN;
        if (std::sqrt(rk2) <= sp.tol * bn) break;
      }
      if (kused == 0) break;
      QCD_TRY(fgcr_backsub(w.d_a1, w.d_a2, w.d_cr, kused, sp.nkv, w.d_gam, s));
      QCD_TRY(blas_multi_axpy(c, phi_p.data(), kused, w.d_gam, (double*)x.data, s));
      QCD_TRY(residual64(c, b, x, w.r, w.d_rn + sp.nkv, s));
      double nrn2 = 0;
      QCD_TRY(read_scalar(w, w.d_rn + sp.nkv, &nrn2, s));
      ++inf.restarts;
      const double nrn = std::sqrt(nrn2);
      if (!(nrn == nrn)) return QCD_NAN;
      slow_cycles = nrn > 0.999 * rn ? slow_cycles + 1 : 0;
      rn = nrn;
      inf.true_residual = rn / bn;
      if (slow_cycles >= 3 && rn > sp.tol * bn) return QCD_STAGNATED;
    }
    return rn <= sp.tol * bn ? QCD_OK : QCD_NOT_CONVERGED;
  };
  st = run();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  inf.time_ms = ms;
  return finish(st);
}

void workspace_free(qcd_ctx* c) {
  Workspace* w = c->ws;
  if (!w) return;
  rec_free(w->sap.rho);
  rec_free(w->sap.psi);
  if (w->sap.faces) cudaFree(w->sap.faces);
  rec_free(w->b);
  rec_free(w->x);
  rec_free(w->r);
  rec_free(w->rho);
  rec_free(w->tmp64);
  rec_free(w->lo_in);
  rec_free(w->lo_out);
  for (auto& r : w->phi) rec_free(r);
  for (auto& r : w->chi) rec_free(r);
  cudaFree(w->d_a1);
  cudaFree(w->d_a2);
  cudaFree(w->d_cr);
  cudaFree(w->d_rn);
  cudaFree(w->d_gam);
  cudaFree(w->d_gs);
  if (w->h_pin) cudaFreeHost(w->h_pin);
  delete w;
  c->ws = nullptr;
}

}  // namespace qcd
