// Small dense complex linear algebra on the host for the FGMRES-DR cycle
// ends (Sec. 4: least squares on the Arnoldi matrix H, harmonic Ritz pairs,
// orthonormal basis of the deflation subspace).  Sizes are the Krylov cycle
// length (<= 64), so plain textbook algorithms suffice: Householder QR, LU
// with partial pivoting, Hessenberg reduction plus shifted QR iterations
// (Wilkinson shift, Givens rotations) to the complex Schur form, and
// eigenvectors by back substitution on the triangular factor.
#include <algorithm>
#include <cmath>

#include "smalldense.h"

namespace qcd {
namespace dense {

static double nrm(const cd* x, int n) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += std::norm(x[i]);
  return std::sqrt(s);
}

// Householder vector of x (length n): H = I - 2 v v^H maps x to alpha e_1
// with alpha = -exp(i arg x_0) |x|; v normalised.  Returns false if x = 0.
static bool householder(const cd* x, int n, std::vector<cd>& v, cd& alpha) {
  const double xn = nrm(x, n);
  v.assign(x, x + n);
  if (xn == 0) return false;
  const cd ph = std::abs(x[0]) > 0 ? x[0] / std::abs(x[0]) : cd(1, 0);
  alpha = -ph * xn;
  v[0] -= alpha;
  const double vn = nrm(v.data(), n);
  if (vn == 0) return false;
  for (auto& e : v) e /= vn;
  return true;
}

void qr_thin(const Mat& A, Mat& Q, Mat& R) {
  const int m = A.r, n = A.c;
  Mat W = A;
  std::vector<std::vector<cd>> vs(n);
  std::vector<bool> used(n, false);
  std::vector<cd> v;
  for (int k = 0; k < n && k < m; ++k) {
    cd alpha;
    if (!householder(&W(k, k), m - k, v, alpha)) continue;
    for (int j = k; j < n; ++j) {  // W[k:, j] -= 2 v (v^H W[k:, j])
      cd s = 0;
      for (int i = 0; i < m - k; ++i) s += std::conj(v[i]) * W(k + i, j);
      s *= 2.0;
      for (int i = 0; i < m - k; ++i) W(k + i, j) -= s * v[i];
    }
    vs[k] = v;
    used[k] = true;
  }
  R = Mat(n, n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= j && i < m; ++i) R(i, j) = W(i, j);
  // Q = H_0 H_1 ... H_{n-1} applied to the first n columns of the identity
  Q = Mat(m, n);
  for (int j = 0; j < n; ++j) Q(j, j) = 1;
  for (int k = std::min(n, m) - 1; k >= 0; --k) {
    if (!used[k]) continue;
    const std::vector<cd>& u = vs[k];
    for (int j = 0; j < n; ++j) {
      cd s = 0;
      for (int i = 0; i < m - k; ++i) s += std::conj(u[i]) * Q(k + i, j);
      s *= 2.0;
      for (int i = 0; i < m - k; ++i) Q(k + i, j) -= s * u[i];
    }
  }
}

bool lstsq(const Mat& A, const std::vector<cd>& c, std::vector<cd>& y, double* res) {
  const int m = A.r, n = A.c;
  Mat Q, R;
  qr_thin(A, Q, R);
  std::vector<cd> qc(n, 0);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) qc[j] += std::conj(Q(i, j)) * c[i];
  y.assign(n, 0);
  for (int i = n - 1; i >= 0; --i) {
    cd s = qc[i];
    for (int j = i + 1; j < n; ++j) s -= R(i, j) * y[j];
    if (std::abs(R(i, i)) == 0) return false;
    y[i] = s / R(i, i);
  }
  if (res) {  // |c - A y|
    double s = 0;
    for (int i = 0; i < m; ++i) {
      cd t = c[i];
      for (int j = 0; j < n; ++j) t -= A(i, j) * y[j];
      s += std::norm(t);
    }
    *res = std::sqrt(s);
  }
  return true;
}

bool solve(Mat A, std::vector<cd>& b) {
  const int n = A.r;
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A(i, k)) > std::abs(A(p, k))) p = i;
    if (std::abs(A(p, k)) == 0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      const cd l = A(i, k) / A(k, k);
      for (int j = k; j < n; ++j) A(i, j) -= l * A(k, j);
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cd s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A(i, j) * b[j];
    b[i] = s / A(i, i);
  }
  return true;
}

// Givens rotation [c s; -conj(s) c] (c real) with G [a; b] = [r; 0]
static void givens(cd a, cd b, double& c, cd& s) {
  const double aa = std::abs(a), bb = std::abs(b);
  if (bb == 0) {
    c = 1;
    s = 0;
    return;
  }
  if (aa == 0) {
    c = 0;
    s = std::conj(b) / bb;
    return;
  }
  const double r = std::hypot(aa, bb);
  c = aa / r;
  s = (a / aa) * std::conj(b) / r;
}

bool eig(const Mat& A0, std::vector<cd>& w, Mat& V) {
  const int n = A0.r;
  Mat H = A0;
  Mat Z(n, n);
  for (int i = 0; i < n; ++i) Z(i, i) = 1;
  // Hessenberg reduction: H = Z^H A Z
  std::vector<cd> v;
  for (int k = 0; k + 2 < n; ++k) {
    cd alpha;
    if (!householder(&H(k + 1, k), n - k - 1, v, alpha)) continue;
    const int l = n - k - 1;
    for (int j = 0; j < n; ++j) {  // left: rows k+1.. of every column
      cd s = 0;
      for (int i = 0; i < l; ++i) s += std::conj(v[i]) * H(k + 1 + i, j);
      s *= 2.0;
      for (int i = 0; i < l; ++i) H(k + 1 + i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {  // right: columns k+1.. of every row
      cd s = 0;
      for (int j = 0; j < l; ++j) s += H(i, k + 1 + j) * v[j];
      s *= 2.0;
      for (int j = 0; j < l; ++j) H(i, k + 1 + j) -= s * std::conj(v[j]);
    }
    for (int i = 0; i < n; ++i) {  // Z = Z H_k
      cd s = 0;
      for (int j = 0; j < l; ++j) s += Z(i, k + 1 + j) * v[j];
      s *= 2.0;
      for (int j = 0; j < l; ++j) Z(i, k + 1 + j) -= s * std::conj(v[j]);
    }
    for (int i = k + 2; i < n; ++i) H(i, k) = 0;
  }
  // shifted QR iterations to the Schur form T = Z^H A Z (upper triangular)
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0, since = 0;
  std::vector<double> cs(n);
  std::vector<cd> sn(n);
  while (hi > 0) {
    if (++iter > 100 * n) return false;
    int lo = hi;
    while (lo > 0) {
      const double sc = std::abs(H(lo, lo)) + std::abs(H(lo - 1, lo - 1));
      if (std::abs(H(lo, lo - 1)) <= eps * (sc > 0 ? sc : 1.0)) {
        H(lo, lo - 1) = 0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // one eigenvalue converged
      --hi;
      since = 0;
      continue;
    }
    // Wilkinson shift from the trailing 2x2 block, exceptional shifts when slow
    cd sigma;
    ++since;
    if (since % 11 == 10) {
      sigma = H(hi, hi) + cd(std::abs(H(hi, hi - 1)), 0);
    } else {
      const cd a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
      const cd tr = a + d, det = a * d - b * c;
      const cd disc = std::sqrt(tr * tr - 4.0 * det);
      const cd l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
      sigma = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
    }
    for (int i = lo; i <= hi; ++i) H(i, i) -= sigma;
    for (int i = lo; i < hi; ++i) {  // left rotations: H <- G H
      givens(H(i, i), H(i + 1, i), cs[i], sn[i]);
      for (int j = i; j < n; ++j) {
        const cd x = H(i, j), y = H(i + 1, j);
        H(i, j) = cs[i] * x + sn[i] * y;
        H(i + 1, j) = -std::conj(sn[i]) * x + cs[i] * y;
      }
    }
    for (int i = lo; i < hi; ++i) {  // right rotations: H <- H G^H, Z <- Z G^H
      const int top = std::min(i + 2, hi);
      for (int r = 0; r <= top; ++r) {
        const cd x = H(r, i), y = H(r, i + 1);
        H(r, i) = cs[i] * x + std::conj(sn[i]) * y;
        H(r, i + 1) = -sn[i] * x + cs[i] * y;
      }
      for (int r = 0; r < n; ++r) {
        const cd x = Z(r, i), y = Z(r, i + 1);
        Z(r, i) = cs[i] * x + std::conj(sn[i]) * y;
        Z(r, i + 1) = -sn[i] * x + cs[i] * y;
      }
    }
    for (int i = lo; i <= hi; ++i) H(i, i) += sigma;
  }
  // eigenvectors of the triangular T by back substitution, then V = Z X
  w.resize(n);
  for (int k = 0; k < n; ++k) w[k] = H(k, k);
  double tn = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= j; ++i) tn = std::max(tn, std::abs(H(i, j)));
  const double small = eps * (tn > 0 ? tn : 1.0);
  V = Mat(n, n);
  std::vector<cd> x(n);
  for (int k = 0; k < n; ++k) {
    std::fill(x.begin(), x.end(), cd(0));
    x[k] = 1;
    for (int j = k - 1; j >= 0; --j) {
      cd s = 0;
      for (int l = j + 1; l <= k; ++l) s += H(j, l) * x[l];
      cd d = H(j, j) - w[k];
      if (std::abs(d) < small) d = small;
      x[j] = -s / d;
    }
    double xn = 0;
    for (int i = 0; i < n; ++i) {
      cd s = 0;
      for (int l = 0; l <= k; ++l) s += Z(i, l) * x[l];
      V(i, k) = s;
      xn += std::norm(s);
    }
    xn = std::sqrt(xn);
    for (int i = 0; i < n; ++i) V(i, k) /= xn;
  }
  return true;
}

}  // namespace dense
}  // namespace qcd
