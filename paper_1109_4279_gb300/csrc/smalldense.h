// Small dense complex matrices on the host (column-major) and the few
// factorisations the FGMRES-DR cycle ends need.
#pragma once
#include <complex>
#include <vector>

namespace qcd {
namespace dense {

typedef std::complex<double> cd;

struct Mat {
  int r = 0, c = 0;
  std::vector<cd> a;
  Mat() = default;
  Mat(int rows, int cols) : r(rows), c(cols), a((size_t)rows * cols, cd(0)) {}
  cd& operator()(int i, int j) { return a[(size_t)i + (size_t)j * r]; }
  const cd& operator()(int i, int j) const { return a[(size_t)i + (size_t)j * r]; }
};

// thin QR of an m x n matrix (m >= n) by Householder reflections: A = Q R,
// Q m x n with orthonormal columns, R n x n upper triangular; the leading j
// columns of Q span the leading j columns of A
void qr_thin(const Mat& A, Mat& Q, Mat& R);
// y = argmin |c - A y| (m >= n, full column rank); res (optional) = |c - A y|
bool lstsq(const Mat& A, const std::vector<cd>& c, std::vector<cd>& y, double* res);
// A x = b in place (LU with partial pivoting); false if A is singular
bool solve(Mat A, std::vector<cd>& b);
// eigenvalues w and unit right eigenvectors (columns of V) of a general
// complex n x n matrix; false if the QR iterations do not converge
bool eig(const Mat& A, std::vector<cd>& w, Mat& V);

}  // namespace dense
}  // namespace qcd
