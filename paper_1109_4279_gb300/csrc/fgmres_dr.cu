// Flexible GMRES with deflated restarts (Sec. 4: "FGMRES-DR"; the flexible
// generalisation of GMRES-DR), preconditioned by SAP, FP64 recursion.
//
// A cycle of length m builds the flexible Arnoldi relation D Z = V Hbar:
//   z_j = M_SAP v_j;  w = D z_j;  w -= V (V^H w) (classical Gram-Schmidt, a
//   second pass decided on the device);  v_{j+1} = w / |w|.
// After every step the host reads H's new column and solves the small least
// squares problem min |c - Hbar y|, whose residual is the residual norm of the
// cycle's iterate; the cycle ends at the tolerance or after m steps, when
// x += Z y and the true FP64 residual b - D x is recomputed.  Unless converged,
// the next cycle starts from the harmonic Ritz vectors of the k smallest
// harmonic Ritz values of (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T) together with
// the residual coordinates c - Hbar y: their orthonormal basis Q (QR on the
// host) gives V <- V Q, Z <- Z Q_k, Hbar <- Q^H Hbar Q_k and c <- Q^H (c - Hbar y),
// and the Arnoldi steps continue from column k (Sec. 4: "this subspace,
// augmented with the residue, becomes the initial Krylov subspace for the
// subsequent restart").
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "smalldense.h"

namespace qcd {

using dense::cd;
using dense::Mat;

void dr_release(Workspace& w) {
  for (auto* v : {&w.drV, &w.drT})
    for (auto& r : *v) rec_free(r);
  w.drV.clear();
  w.drT.clear();
  if (w.h_hcol) cudaFreeHost(w.h_hcol);
  w.h_hcol = nullptr;
  if (w.d_hnorm) cudaFree(w.d_hnorm);
  w.d_hnorm = nullptr;
}

static int dr_prepare(qcd_ctx* c, Workspace& w, const qcd_solver_params& sp, cudaStream_t s) {
  QCD_TRY(ws_prepare(c, w, sp, s));  // b, x, r, phi (= Z), chi (= V_0..V_{m-1}), scalars, SAP fields
  const int k = sp.ndefl;
  while ((int)w.drV.size() < 1) {
    w.drV.emplace_back();
    QCD_TRY(rec_alloc(w.drV.back(), P64, 24, c->V));
  }
  while ((int)w.drT.size() < k + 1) {
    w.drT.emplace_back();
    QCD_TRY(rec_alloc(w.drT.back(), P64, 24, c->V));
  }
  // pinned column buffer: pass-1 and pass-2 coefficients (2 x 2 (m + 1)) and
  // the subdiagonal; device buffer: subdiagonals, then restart coefficients
  if (!w.h_hcol) QCD_CUDA(cudaMallocHost(&w.h_hcol, sizeof(double) * (4 * 65 + 8)));
  if (!w.d_hnorm) QCD_CUDA(cudaMalloc(&w.d_hnorm, sizeof(double) * (65 + 2 * 65 * 65)));
  return QCD_OK;
}

// solve one problem; p.c, p.w, p.s, p.b, p.x set by the caller
static int dr_solve(Problem& p, const qcd_solver_params& sp) {
  qcd_ctx* c = p.c;
  Workspace& w = *p.w;
  cudaStream_t s = p.s;
  const int m = sp.nkv, k = sp.ndefl;
  const size_t dsz = sizeof(double);
  memset(&p.info, 0, sizeof(p.info));
  p.status = QCD_OK;
  int st = dr_prepare(c, w, sp, s);
  if (st != QCD_OK) return p.status = st;
  QCD_CUDA(cudaMemsetAsync(c->d_scalars + 128, 0, dsz, s));  // SAP staging time-out flag
  // basis handles (slots of the workspace; restarts swap their contents)
  std::vector<Rec*> V(m + 1), Z(m), T(k + 1);
  for (int j = 0; j < m; ++j) V[j] = &w.chi[j];
  V[m] = &w.drV[0];
  for (int j = 0; j < m; ++j) Z[j] = &w.phi[j];
  for (int i = 0; i <= k; ++i) T[i] = &w.drT[i];
  double* d_q = w.d_hnorm + 65;  // restart coefficients, complex, column i at 2 (m + 1) i
  const int ld = sp.nkv;

  // |b|, |x0|, r = b - D x0 (or b)
  QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)p.b.data, w.d_rn + ld, s));
  QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)p.x.data, w.d_rn + ld + 3, s));
  QCD_CUDA(cudaMemcpyAsync(w.h_pin + ld, w.d_rn + ld, 4 * dsz, cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  if (w.h_pin[ld + 3] == 0.0) {
    QCD_CUDA(cudaMemcpyAsync(w.r.data, p.b.data, w.r.bytes, cudaMemcpyDeviceToDevice, s));
    QCD_CUDA(cudaMemcpyAsync(w.d_rn + ld + 1, w.d_rn + ld, dsz, cudaMemcpyDeviceToDevice, s));
  } else {
    QCD_TRY(residual64(c, w.d_part, p.b, p.x, w.r, w.d_rn + ld + 1, s));
  }
  QCD_CUDA(cudaMemcpyAsync(w.h_pin + ld + 1, w.d_rn + ld + 1, dsz, cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  const double bn2 = w.h_pin[ld], rn2 = w.h_pin[ld + 1];
  if (!(bn2 == bn2) || std::isinf(bn2) || !(rn2 == rn2)) return p.status = QCD_NAN;
  if (bn2 == 0.0) {
    QCD_CUDA(cudaMemsetAsync(p.x.data, 0, p.x.bytes, s));
    return QCD_OK;
  }
  p.bn = std::sqrt(bn2);
  p.rn = std::sqrt(rn2);
  p.info.true_residual = p.rn / p.bn;
  if (p.rn <= sp.tol * p.bn) return QCD_OK;

  // v_0 = r / |r| (gs_normalise reads |r|^2 at gs[1])
  auto start_from_residual = [&](const double* d_rn2) -> int {
    QCD_CUDA(cudaMemcpyAsync(V[0]->data, w.r.data, w.r.bytes, cudaMemcpyDeviceToDevice, s));
    return blas_gs_normalise(c, (double*)V[0]->data, d_rn2 - 1, 0, w.d_hnorm, s);
  };
  QCD_TRY(start_from_residual(w.d_rn + ld + 1));
  Mat H(m + 1, m);
  std::vector<cd> cvec(m + 1, cd(0));
  cvec[0] = p.rn;
  int j0 = 0;
  p.slow = 0;
  for (;;) {
    if (p.info.restarts >= sp.max_restarts) return p.status = QCD_NOT_CONVERGED;
    // ---- Arnoldi steps j0 .. m-1
    int jend = m;
    std::vector<cd> y;
    for (int j = j0; j < m; ++j) {
      if (sp.precond == QCD_PRECOND_SAP) {
        QCD_TRY(sap_apply(c, w.sap, *V[j], *Z[j], sp.ncy, sp.nmr, sp.sap_prec, s));
      } else {
        QCD_CUDA(cudaMemcpyAsync(Z[j]->data, V[j]->data, V[j]->bytes, cudaMemcpyDeviceToDevice, s));
      }
      double* wv = (double*)V[j + 1]->data;
      QCD_TRY(dirac_apply(c, *Z[j], *V[j + 1], 0, s));
      const double* vp[65];
      for (int i = 0; i <= j; ++i) vp[i] = (const double*)V[i]->data;
      double* a1 = w.d_a1 + 2 * (size_t)j * ld;
      double* a2 = w.d_a2 + 2 * (size_t)j * ld;
      double* gs = w.d_gs + 8 * (size_t)j;
      // (the norm kernels also form (w, v_0), which Arnoldi does not use)
      QCD_TRY(blas_multidot<double>(c, w.d_part, vp, j + 1, wv, a1, s, nullptr, gs));
      QCD_TRY(blas_axpy_norm_dot<double>(c, w.d_part, vp, j + 1, a1, wv, vp[0], gs + 1, s));
      QCD_TRY(blas_multidot<double>(c, w.d_part, vp, j + 1, wv, a2, s, gs));
      QCD_TRY(blas_axpy_norm_dot<double>(c, w.d_part, vp, j + 1, a2, wv, vp[0], gs + 4, s, gs));
      QCD_TRY(blas_gs_normalise(c, wv, gs, 1, w.d_hnorm + j, s));
      double* hc = w.h_hcol;
      QCD_CUDA(cudaMemcpyAsync(hc, a1, 2 * (j + 1) * dsz, cudaMemcpyDeviceToHost, s));
      QCD_CUDA(cudaMemcpyAsync(hc + 2 * 65, a2, 2 * (j + 1) * dsz, cudaMemcpyDeviceToHost, s));
      QCD_CUDA(cudaMemcpyAsync(hc + 4 * 65, w.d_hnorm + j, dsz, cudaMemcpyDeviceToHost, s));
      QCD_CUDA(cudaStreamSynchronize(s));
      ++p.info.iterations;
      for (int i = 0; i <= j; ++i) H(i, j) = cd(hc[2 * i] + hc[2 * 65 + 2 * i], hc[2 * i + 1] + hc[2 * 65 + 2 * i + 1]);
      H(j + 1, j) = hc[4 * 65];
      if (!(hc[4 * 65] == hc[4 * 65])) return p.status = QCD_NAN;
      // least squares over the columns built so far
      Mat Hs(j + 2, j + 1);
      for (int b = 0; b <= j; ++b)
        for (int a = 0; a <= j + 1; ++a) Hs(a, b) = H(a, b);
      std::vector<cd> cs(cvec.begin(), cvec.begin() + j + 2);
      double res = 0;
      if (!dense::lstsq(Hs, cs, y, &res)) return p.status = QCD_STAGNATED;
      if (res <= sp.tol * p.bn || hc[4 * 65] == 0.0) {
        jend = j + 1;
        break;
      }
    }
    // ---- x += Z y; true FP64 residual
    std::vector<double> yd(2 * jend);
    for (int i = 0; i < jend; ++i) {
      yd[2 * i] = y[i].real();
      yd[2 * i + 1] = y[i].imag();
    }
    QCD_CUDA(cudaMemcpyAsync(w.d_gam, yd.data(), 2 * jend * dsz, cudaMemcpyHostToDevice, s));
    {
      const double* zp[64];
      for (int i = 0; i < jend; ++i) zp[i] = (const double*)Z[i]->data;
      QCD_TRY(blas_multi_axpy<double>(c, zp, jend, w.d_gam, (double*)p.x.data, s));
    }
    QCD_TRY(residual64(c, w.d_part, p.b, p.x, w.r, w.d_rn + ld + 2, s));
    QCD_CUDA(cudaMemcpyAsync(w.h_pin + ld + 2, w.d_rn + ld + 2, dsz, cudaMemcpyDeviceToHost, s));
    QCD_CUDA(cudaMemcpyAsync(w.h_pin + ld + 3, (const double*)(c->d_scalars + 128), dsz, cudaMemcpyDeviceToHost, s));
    QCD_CUDA(cudaStreamSynchronize(s));
    ++p.info.restarts;
    int sap_err = 0;
    memcpy(&sap_err, w.h_pin + ld + 3, sizeof(int));
    if (sap_err) return p.status = QCD_ERR_TIMEOUT;
    const double nrn = std::sqrt(w.h_pin[ld + 2]);
    if (!(nrn == nrn)) return p.status = QCD_NAN;
    p.slow = nrn > 0.999 * p.rn ? p.slow + 1 : 0;
    p.rn = nrn;
    p.info.true_residual = nrn / p.bn;
    if (nrn <= sp.tol * p.bn) return QCD_OK;
    if (p.slow >= 3) return p.status = QCD_STAGNATED;
    // ---- restart: deflated (harmonic Ritz vectors + residual) or plain
    std::vector<cd> sres(jend + 1);
    for (int a = 0; a <= jend; ++a) {
      cd t = cvec[a];
      for (int b = 0; b < jend; ++b) t -= H(a, b) * y[b];
      sres[a] = t;
    }
    bool deflated = false;
    Mat Q;
    if (k > 0 && jend > k && std::abs(H(jend, jend - 1)) > 0) {
      Mat Hm(jend, jend);
      for (int b = 0; b < jend; ++b)
        for (int a = 0; a < jend; ++a) Hm(a, b) = H(a, b);
      Mat HmH(jend, jend);
      for (int b = 0; b < jend; ++b)
        for (int a = 0; a < jend; ++a) HmH(a, b) = std::conj(Hm(b, a));
      std::vector<cd> f(jend, cd(0));
      f[jend - 1] = 1;
      std::vector<cd> theta;
      Mat G = Hm, gv;
      if (dense::solve(HmH, f)) {
        const double h2 = std::norm(H(jend, jend - 1));
        for (int a = 0; a < jend; ++a) G(a, jend - 1) += h2 * f[a];
        if (dense::eig(G, theta, gv)) {
          std::vector<int> order(jend);
          std::iota(order.begin(), order.end(), 0);
          std::stable_sort(order.begin(), order.end(),
                           [&](int a, int b) { return std::abs(theta[a]) < std::abs(theta[b]); });
          Mat P(jend + 1, k + 1);
          for (int i = 0; i < k; ++i)
            for (int a = 0; a < jend; ++a) P(a, i) = gv(a, order[i]);
          for (int a = 0; a <= jend; ++a) P(a, k) = sres[a];
          Mat R;
          dense::qr_thin(P, Q, R);
          deflated = true;
          for (int i = 0; i <= k && deflated; ++i)
            if (!(std::abs(R(i, i)) > 1e-14 * std::abs(R(0, 0)))) deflated = false;  // dependent columns
        }
      }
    }
    if (deflated) {
      // coefficients to the device: column i of Q at 2 (jend + 1) i
      std::vector<double> qd(2 * (size_t)(jend + 1) * (k + 1));
      for (int i = 0; i <= k; ++i)
        for (int a = 0; a <= jend; ++a) {
          qd[2 * ((size_t)i * (jend + 1) + a)] = Q(a, i).real();
          qd[2 * ((size_t)i * (jend + 1) + a) + 1] = Q(a, i).imag();
        }
      QCD_CUDA(cudaMemcpyAsync(d_q, qd.data(), qd.size() * dsz, cudaMemcpyHostToDevice, s));
      const double* vp[65];
      for (int a = 0; a <= jend; ++a) vp[a] = (const double*)V[a]->data;
      for (int i = 0; i <= k; ++i) {  // T_i = sum_a Q(a, i) V_a
        QCD_CUDA(cudaMemsetAsync(T[i]->data, 0, T[i]->bytes, s));
        QCD_TRY(blas_multi_axpy<double>(c, vp, jend + 1, d_q + 2 * (size_t)i * (jend + 1), (double*)T[i]->data, s));
      }
      for (int i = 0; i <= k; ++i) std::swap(*V[i], *T[i]);
      const double* zp[64];
      for (int a = 0; a < jend; ++a) zp[a] = (const double*)Z[a]->data;
      for (int i = 0; i < k; ++i) {  // T_i = sum_{a < jend} Q(a, i) Z_a
        QCD_CUDA(cudaMemsetAsync(T[i]->data, 0, T[i]->bytes, s));
        QCD_TRY(blas_multi_axpy<double>(c, zp, jend, d_q + 2 * (size_t)i * (jend + 1), (double*)T[i]->data, s));
      }
      for (int i = 0; i < k; ++i) std::swap(*Z[i], *T[i]);
      // Hbar <- Q^H Hbar Q_k, c <- Q^H s
      Mat HQ(jend + 1, k);
      for (int i = 0; i < k; ++i)
        for (int a = 0; a <= jend; ++a) {
          cd t = 0;
          for (int b = 0; b < jend; ++b) t += H(a, b) * Q(b, i);
          HQ(a, i) = t;
        }
      Mat Hn(k + 1, k);
      for (int i = 0; i < k; ++i)
        for (int r = 0; r <= k; ++r) {
          cd t = 0;
          for (int a = 0; a <= jend; ++a) t += std::conj(Q(a, r)) * HQ(a, i);
          Hn(r, i) = t;
        }
      std::vector<cd> cn(k + 1, cd(0));
      for (int r = 0; r <= k; ++r)
        for (int a = 0; a <= jend; ++a) cn[r] += std::conj(Q(a, r)) * sres[a];
      H = Mat(m + 1, m);
      for (int i = 0; i < k; ++i)
        for (int r = 0; r <= k; ++r) H(r, i) = Hn(r, i);
      std::fill(cvec.begin(), cvec.end(), cd(0));
      for (int r = 0; r <= k; ++r) cvec[r] = cn[r];
      j0 = k;
    } else {
      QCD_TRY(start_from_residual(w.d_rn + ld + 2));
      H = Mat(m + 1, m);
      std::fill(cvec.begin(), cvec.end(), cd(0));
      cvec[0] = p.rn;
      j0 = 0;
    }
  }
}

int fgmres_dr_batch(std::vector<Problem>& probs, const qcd_solver_params& sp) {
  NvtxRange nv("fgmres_dr");
  if (sp.nkv < 2 || sp.nkv > 64 || sp.ndefl < 0 || sp.ndefl >= sp.nkv || !(sp.tol > 0) || sp.max_restarts < 1)
    return QCD_ERR_ARG;
  if (sp.outer_prec != P64) return QCD_ERR_UNSUPPORTED;
  if (sp.precond != QCD_PRECOND_NONE && sp.precond != QCD_PRECOND_SAP) return QCD_ERR_ARG;
  if (sp.precond == QCD_PRECOND_SAP && (sp.ncy < 1 || sp.nmr < 0 || sp.sap_prec < P64 || sp.sap_prec > PB16))
    return QCD_ERR_ARG;
  int first = QCD_OK;
  for (auto& p : probs) {
    if (!p.c->clover_built) {
      p.status = QCD_ERR_STATE;
    } else {
      int st = dr_solve(p, sp);
      if (st != QCD_OK && p.status == QCD_OK) p.status = st;
      // restarts permuted the fields behind the workspace slots: captured FGCR
      // iteration graphs refer to the old pointers
      for (auto g : p.w->graphs)
        if (g) cudaGraphExecDestroy(g);
      p.w->graphs.clear();
      p.w->graph_warm.clear();
      p.w->graph_key = GraphKey();
    }
    p.info.status = p.status;
    if (p.status != QCD_OK && first == QCD_OK) first = p.status;
  }
  return first;
}

}  // namespace qcd
