// CG on the normal equations D^+ D x = D^+ b, FP64 (Sec. 4: "automatic
// switching to CG for the most difficult cases").  Textbook CG on the
// Hermitian positive definite D^+ D, with the FP64 operator and its adjoint:
//   r = D^+ (b - D x);  p = r
//   repeat: t = D p;  alpha = |r|^2 / |t|^2;  x += alpha p;  r -= alpha D^+ t;
//           p = r + (|r_new|^2 / |r|^2) p
// The coefficients stay on the device (no host synchronisation per
// iteration); every 16 iterations the true residual b - D x is recomputed
// and read back to decide convergence against |b - D x| <= tol |b|.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace qcd {

void cg_release(Workspace& w) {
  for (auto& r : w.cgv) rec_free(r);
  w.cgv.clear();
  if (w.d_cg) cudaFree(w.d_cg);
  w.d_cg = nullptr;
  if (w.h_cg) cudaFreeHost(w.h_cg);
  w.h_cg = nullptr;
}

static int cg_prepare(qcd_ctx* c, Workspace& w, size_t nvec = 4) {
  if (!w.r.data) QCD_TRY(rec_alloc(w.r, P64, 24, c->V));
  while (w.cgv.size() < nvec) {
    w.cgv.emplace_back();
    QCD_TRY(rec_alloc(w.cgv.back(), P64, 24, c->V));
  }
  if (!w.d_part) {
    if (cudaMalloc(&w.d_part, sizeof(double) * partials_for(c->V)) != cudaSuccess) {
      cudaGetLastError();
      w.d_part = nullptr;
      return QCD_ERR_NOMEM;
    }
    w.ps = (long long)partials_for(c->V);
  }
  if (!w.d_cg) QCD_CUDA(cudaMalloc(&w.d_cg, sizeof(double) * 8));
  if (!w.h_cg) QCD_CUDA(cudaMallocHost(&w.h_cg, sizeof(double) * 8));
  return QCD_OK;
}

static const int kCheckEvery = 16;

// d_cg: [0] |b|^2, [1] |b - D x|^2, [2], [3] |r|^2 (alternating), [4] |D p|^2
static int cg_solve(Problem& p, const qcd_solver_params& sp, bool fallback) {
  qcd_ctx* c = p.c;
  Workspace& w = *p.w;
  cudaStream_t s = p.s;
  const size_t dsz = sizeof(double);
  if (!fallback) memset(&p.info, 0, sizeof(p.info));
  p.status = QCD_OK;
  QCD_TRY(cg_prepare(c, w));
  Rec& R = w.cgv[0];
  Rec& P = w.cgv[1];
  Rec& T = w.cgv[2];
  Rec& Q = w.cgv[3];
  double* dc = w.d_cg;
  double* hc = w.h_cg;
  QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)p.b.data, dc + 0, s));
  QCD_TRY(residual64(c, w.d_part, p.b, p.x, w.r, dc + 1, s));
  QCD_TRY(dirac_apply(c, w.r, R, 1, s));
  QCD_CUDA(cudaMemcpyAsync(P.data, R.data, R.bytes, cudaMemcpyDeviceToDevice, s));
  QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)R.data, dc + 2, s));
  QCD_CUDA(cudaMemcpyAsync(hc, dc, 3 * dsz, cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  if (!(hc[0] == hc[0]) || !(hc[1] == hc[1]) || !(hc[2] == hc[2])) return p.status = QCD_NAN;
  if (hc[0] == 0.0) {
    QCD_CUDA(cudaMemsetAsync(p.x.data, 0, p.x.bytes, s));
    p.info.true_residual = 0;
    return QCD_OK;
  }
  p.bn = std::sqrt(hc[0]);
  p.rn = std::sqrt(hc[1]);
  p.info.true_residual = p.rn / p.bn;
  if (p.rn <= sp.tol * p.bn) return QCD_OK;
  const int max_it = sp.cg_max_iter > 0 ? sp.cg_max_iter : 20000;
  for (int it = 1; it <= max_it; ++it) {
    double* rr = dc + 2 + ((it - 1) & 1);
    double* rr_new = dc + 2 + (it & 1);
    QCD_TRY(dirac_apply(c, P, T, 0, s));
    QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)T.data, dc + 4, s));
    QCD_TRY(dirac_apply(c, T, Q, 1, s));
    QCD_TRY(blas_cg_update(c, w.d_part, (double*)p.x.data, (double*)R.data, (const double*)P.data,
                           (const double*)Q.data, rr, dc + 4, rr_new, s));
    QCD_TRY(blas_cg_direction(c, (double*)P.data, (const double*)R.data, rr_new, rr, s));
    p.info.cg_iterations = it;
    if (it % kCheckEvery == 0 || it == max_it) {
      QCD_TRY(residual64(c, w.d_part, p.b, p.x, w.r, dc + 1, s));
      QCD_CUDA(cudaMemcpyAsync(hc, dc, 5 * dsz, cudaMemcpyDeviceToHost, s));
      QCD_CUDA(cudaStreamSynchronize(s));
      if (!(hc[1] == hc[1])) return p.status = QCD_NAN;
      p.rn = std::sqrt(hc[1]);
      p.info.true_residual = p.rn / p.bn;
      if (p.rn <= sp.tol * p.bn) return QCD_OK;
    }
  }
  return p.status = QCD_NOT_CONVERGED;
}

// out = a - b over n doubles
__global__ void __launch_bounds__(256) sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b,
                                                  double2* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 u = a[i], v = b[i];
    out[i] = make_double2(u.x - v.x, u.y - v.y);
  }
}

static int sub(qcd_ctx* c, const Rec& a, const Rec& b, const Rec& out, cudaStream_t s) {
  const long long n = c->V * 12;
  const long long blocks = (n + 255) / 256;
  sub_kernel<<<(unsigned)(blocks < 4 * 152 * 8 ? blocks : 4 * 152 * 8), 256, 0, s>>>(
      (const double2*)a.data, (const double2*)b.data, (double2*)out.data, n);
  QCD_LAUNCHED();
  return QCD_OK;
}

// Even/odd-preconditioned CG (the global even/odd split that goes with the
// CG of Sec. 4).  With D = [[A_ee, H_eo], [H_oe, A_oo]]:
//   bhat_e = b_e - H_eo A_oo^-1 b_o,  Dhat = A_ee - H_eo A_oo^-1 H_oe,
//   CG on Dhat^+ Dhat x_e = Dhat^+ bhat_e (the steps of cg_solve),
//   x_o = A_oo^-1 (b_o - H_oe x_e).
// The whole system's residual is (bhat_e - Dhat x_e, 0), so convergence is
// checked on the even sites every 16 iterations, and b - D x is recomputed
// in FP64 after the reconstruction.  The vectors are full fields whose odd
// sites stay zero, so the FP64 vector kernels serve unchanged.
// d_cg as in cg_solve, [1] |bhat - Dhat x|^2.
static int cg_eo_solve(Problem& p, const qcd_solver_params& sp, bool fallback) {
  qcd_ctx* c = p.c;
  Workspace& w = *p.w;
  cudaStream_t s = p.s;
  const size_t dsz = sizeof(double);
  if (!fallback) memset(&p.info, 0, sizeof(p.info));
  p.status = QCD_OK;
  QCD_TRY(cg_prepare(c, w, 6));
  Rec& R = w.cgv[0];
  Rec& P = w.cgv[1];
  Rec& T = w.cgv[2];
  Rec& Q = w.cgv[3];
  Rec& BH = w.cgv[4];
  Rec& TMP = w.cgv[5];
  for (Rec* f : {&R, &P, &T, &Q, &BH}) QCD_CUDA(cudaMemsetAsync(f->data, 0, f->bytes, s));
  double* dc = w.d_cg;
  double* hc = w.h_cg;
  QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)p.b.data, dc + 0, s));
  QCD_TRY(eo_apply(c, p.b, p.b, TMP, 1, 0, 1, 1, 1.0, 0.0, s));   // TMP_o = A_oo^-1 b_o
  QCD_TRY(eo_apply(c, p.b, TMP, BH, 0, 0, 1, 0, 1.0, -1.0, s));  // BH_e = b_e - H_eo TMP_o
  // Schur residual of the initial even part: w.r = bhat - Dhat x
  auto schur_residual = [&]() -> int {
    QCD_TRY(schur_apply(c, p.x, TMP, T, 0, s));
    QCD_TRY(sub(c, BH, T, w.r, s));
    return blas_norm2<double>(c, w.d_part, (const double*)w.r.data, dc + 1, s);
  };
  QCD_TRY(schur_residual());
  QCD_TRY(schur_apply(c, w.r, TMP, R, 1, s));  // R = Dhat^+ (bhat - Dhat x)
  QCD_CUDA(cudaMemcpyAsync(P.data, R.data, R.bytes, cudaMemcpyDeviceToDevice, s));
  QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)R.data, dc + 2, s));
  QCD_CUDA(cudaMemcpyAsync(hc, dc, 3 * dsz, cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  if (!(hc[0] == hc[0]) || !(hc[1] == hc[1]) || !(hc[2] == hc[2])) return p.status = QCD_NAN;
  if (hc[0] == 0.0) {
    QCD_CUDA(cudaMemsetAsync(p.x.data, 0, p.x.bytes, s));
    p.info.true_residual = 0;
    return QCD_OK;
  }
  p.bn = std::sqrt(hc[0]);
  const int max_it = sp.cg_max_iter > 0 ? sp.cg_max_iter : 20000;
  bool done = std::sqrt(hc[1]) <= sp.tol * p.bn;
  for (int it = 1; it <= max_it || done; ++it) {
    if (done) {  // odd sites from the even ones, then the FP64 residual of D x = b
      QCD_TRY(eo_apply(c, p.b, p.x, p.x, 1, 0, 0, 1, 1.0, -1.0, s));
      QCD_TRY(residual64(c, w.d_part, p.b, p.x, w.r, dc + 1, s));
      QCD_CUDA(cudaMemcpyAsync(hc + 1, dc + 1, dsz, cudaMemcpyDeviceToHost, s));
      QCD_CUDA(cudaStreamSynchronize(s));
      if (!(hc[1] == hc[1])) return p.status = QCD_NAN;
      p.rn = std::sqrt(hc[1]);
      p.info.true_residual = p.rn / p.bn;
      if (p.rn <= sp.tol * p.bn) return QCD_OK;
      done = false;  // rounding of the reconstruction: keep iterating
      if (it > max_it) break;
    }
    double* rr = dc + 2 + ((it - 1) & 1);
    double* rr_new = dc + 2 + (it & 1);
    QCD_TRY(schur_apply(c, P, TMP, T, 0, s));
    QCD_TRY(blas_norm2<double>(c, w.d_part, (const double*)T.data, dc + 4, s));
    QCD_TRY(schur_apply(c, T, TMP, Q, 1, s));
    QCD_TRY(blas_cg_update(c, w.d_part, (double*)p.x.data, (double*)R.data, (const double*)P.data,
                           (const double*)Q.data, rr, dc + 4, rr_new, s));
    QCD_TRY(blas_cg_direction(c, (double*)P.data, (const double*)R.data, rr_new, rr, s));
    p.info.cg_iterations += 1;
    if (it % kCheckEvery == 0 || it == max_it) {
      QCD_TRY(schur_residual());
      QCD_CUDA(cudaMemcpyAsync(hc + 1, dc + 1, dsz, cudaMemcpyDeviceToHost, s));
      QCD_CUDA(cudaStreamSynchronize(s));
      if (!(hc[1] == hc[1])) return p.status = QCD_NAN;
      p.info.true_residual = std::sqrt(hc[1]) / p.bn;
      done = std::sqrt(hc[1]) <= sp.tol * p.bn;
      if (it == max_it && !done) break;
    }
  }
  return p.status = QCD_NOT_CONVERGED;
}

int cg_batch(std::vector<Problem>& probs, const qcd_solver_params& sp, bool fallback_only) {
  NvtxRange nv(fallback_only ? "cg_fallback" : "cg");
  if (!(sp.tol > 0)) return QCD_ERR_ARG;
  int first = QCD_OK;
  for (auto& p : probs) {
    if (fallback_only && p.status != QCD_STAGNATED && p.status != QCD_NOT_CONVERGED) continue;
    if (!p.c->clover_built) {
      p.status = QCD_ERR_STATE;
    } else {
      const bool eo = fallback_only ? sp.cg_fallback == 2 : sp.solver == QCD_SOLVER_CG_EO;
      const int st = eo ? cg_eo_solve(p, sp, fallback_only) : cg_solve(p, sp, fallback_only);
      if (st != QCD_OK && p.status == QCD_OK) p.status = st;
    }
    p.info.status = p.status;
    if (p.status != QCD_OK && first == QCD_OK) first = p.status;
  }
  return first;
}

}  // namespace qcd
