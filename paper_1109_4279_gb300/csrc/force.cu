// Fermion force (Sec. 1: the inversions feed the HMC force): for
// L = Re(phi^+ x), x = D^-1 phi, y = D^-+ phi and the link deformation
// U_mu(x) -> exp(i theta_a lambda_a / 2) U_mu(x),
//   F_a(x, mu) = dL/dtheta_a = -Re(y^+ (dD/dtheta_a) x).
//
// Hopping part (the link appears in D at x and at x + mu):
//   F_a = -(eta/4) Im tr[lambda_a (U P1 - P2 U^+)],
//   P1 = sum_s h_s k_s^+,  h = proj_(1-g)(x(x+mu)), k = proj_(1-g)(y(x)),
//   P2 = sum_s h'_s k'_s^+, h' = proj_(1+g)(x(x)),  k' = proj_(1+g)(y(x+mu)),
// where proj keeps the two upper spin components of (1 -+ g_mu) psi (the
// lower two are fixed by them, which folds the spin trace to two terms).
//
// Clover part: with both orientations summed, the clover term equals
// (i c_sw / 16) sum_{rho != sigma} sigma_{rho sigma} (x) Q_{rho sigma}, so
//   F_a = (c_sw / 32) Re tr[lambda_a sum U S]   (sum over the 24 leaf
// occurrences of the link; a daggered occurrence contributes -S U^+), where S
// is the rest of the leaf read cyclically from the link, with
// W_{rho sigma}(z) = X + X^+, X = sum_{s,t} sigma_{rho sigma}[s][t] x_t(z) y_s(z)^+,
// inserted at the leaf's corner z.
#include "internal.h"

namespace qcd {

typedef cpx<double> cd;

struct C3 {
  cd m[3][3];
};

__device__ __forceinline__ C3 c3mul(const C3& a, const C3& b) {
  C3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd v = cmul(a.m[i][0], b.m[0][j]);
      v = cmadd(a.m[i][1], b.m[1][j], v);
      v = cmadd(a.m[i][2], b.m[2][j], v);
      r.m[i][j] = v;
    }
  return r;
}

__device__ __forceinline__ C3 c3dag(const C3& a) {
  C3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[i][j] = conjg(a.m[j][i]);
  return r;
}

__device__ __forceinline__ void c3acc(C3& a, const C3& b, double s) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a.m[i][j] = a.m[i][j] + s * b.m[i][j];
}

// tr(lambda_a M), a = 1..8
__device__ __forceinline__ void trace_lambda(const C3& M, cd t[8]) {
  const double r3 = 0.57735026918962576451;  // 1 / sqrt(3)
  t[0] = M.m[1][0] + M.m[0][1];
  t[1] = mti(M.m[1][0]) + ti(M.m[0][1]);
  t[2] = M.m[0][0] - M.m[1][1];
  t[3] = M.m[2][0] + M.m[0][2];
  t[4] = mti(M.m[2][0]) + ti(M.m[0][2]);
  t[5] = M.m[2][1] + M.m[1][2];
  t[6] = mti(M.m[2][1]) + ti(M.m[1][2]);
  cd d = M.m[0][0] + M.m[1][1] - 2.0 * M.m[2][2];
  t[7] = r3 * d;
}

__device__ __forceinline__ C3 link64(const Geom& g, const double2* U, long long s, int mu) {
  const int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  SU3<double> u = load_link<P64, double>(U, g.Vb, blk, r, mu);
  C3 o;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) o.m[i][j] = u.m[i][j];
  return o;
}

// internal index of x + s_mu mu-hat + s_nu nu-hat (periodic).  Written with
// selects only: no dynamically indexed local arrays, whose copies the
// compiler is free to place in overlapping stack slots.
__device__ __forceinline__ long long shifted(const Geom& g, const int x[4], int mu, int smu, int nu, int snu) {
  int y[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int o = (d == mu ? smu : 0) + (d == nu ? snu : 0);
    y[d] = (x[d] + o + g.L[d]) % g.L[d];
  }
  return internal_index(g, y);
}

// plane index of (rho < sigma): 01 02 03 12 13 23
__device__ __forceinline__ int plane(int a, int b) {
  int r = a < b ? a : b, s = a < b ? b : a;
  return r == 0 ? s - 1 : (r == 1 ? s + 1 : 5);
}

// W_{rho sigma}(z) = X + X^+ for the 6 planes; X = sum_st sigma[s][t] x_t y_s^+.
// sigma_0k = diag(s_k, -s_k), sigma_jk = -eps_jkl diag(s_l, s_l) in the chiral basis.
__global__ void force_w_kernel(Geom g, FieldPtr xf, FieldPtr yf, double2* __restrict__ W) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  Spinor<double> x = load_spinor<P64, double>(xf, g.Vb, blk, r);
  Spinor<double> y = load_spinor<P64, double>(yf, g.Vb, blk, r);
  // O[s][t] = x_t y_s^+ (colour matrices) for s, t in the same chiral block
  for (int p = 0; p < 6; ++p) {
    // the Pauli index l and signs of sigma in the upper / lower chiral block
    int l;
    double su, sl;
    switch (p) {
      case 0: l = 0; su = 1; sl = -1; break;   // 01: sigma_1
      case 1: l = 1; su = 1; sl = -1; break;   // 02: sigma_2
      case 2: l = 2; su = 1; sl = -1; break;   // 03: sigma_3
      case 3: l = 2; su = -1; sl = -1; break;  // 12: -sigma_3
      case 4: l = 1; su = 1; sl = 1; break;    // 13: +sigma_2
      default: l = 0; su = -1; sl = -1; break; // 23: -sigma_1
    }
    C3 X;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) X.m[a][b] = {0, 0};
    for (int ch = 0; ch < 2; ++ch) {
      const double sg = ch == 0 ? su : sl;
      for (int si = 0; si < 2; ++si)
        for (int ti_ = 0; ti_ < 2; ++ti_) {
          // Pauli matrix element [si][ti]
          cd pm;
          if (l == 0) pm = {si != ti_ ? 1.0 : 0.0, 0.0};
          else if (l == 1) pm = {0.0, si == ti_ ? 0.0 : (si == 0 ? -1.0 : 1.0)};
          else pm = {si == ti_ ? (si == 0 ? 1.0 : -1.0) : 0.0, 0.0};
          if (pm.re == 0.0 && pm.im == 0.0) continue;
          pm = sg * pm;
          const int S = 2 * ch + si, T = 2 * ch + ti_;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) X.m[a][b] = cmadd(pm, cmul(x.c[T][a], conjg(y.c[S][b])), X.m[a][b]);
        }
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        cd w = X.m[a][b] + conjg(X.m[b][a]);
        W[(s * 6 + p) * 9 + a * 3 + b] = make_double2(w.re, w.im);
      }
  }
}

__device__ __forceinline__ C3 load_w(const double2* W, long long s, int p) {
  C3 o;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = W[(s * 6 + p) * 9 + k];
    o.m[k / 3][k % 3] = {v.x, v.y};
  }
  return o;
}

// contribution of one plaquette cycle C[0..3] (corners c[0..3]) in which the
// link sits at position p (daggered or not) to M = sum (U S  or  -S U^+)
__device__ void plaquette_terms(const C3 C[4], const long long c[4], int p, bool dag, int pl, const double2* W,
                                C3& M) {
  C3 acc;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) acc.m[i][j] = {0, 0};
  for (int k = 0; k < 4; ++k) {
    // S = C[p+1] ... C[k-1] W(c_k) C[k] ... C[p-1]  (cyclic)
    const int j = (k - p - 1 + 8) & 3;  // links before W
    C3 S;
    bool first = true;
    for (int q = 0; q < 4; ++q) {
      C3 f;
      if (q == j) {
        f = load_w(W, c[k], pl);
      } else {
        const int idx = (p + 1 + (q < j ? q : q - 1)) & 3;
        f = C[idx];
      }
      S = first ? f : c3mul(S, f);
      first = false;
    }
    c3acc(acc, S, 1.0);
  }
  const C3& U = C[p];  // the link as it appears in the cycle (U or U^+)
  if (!dag) {
    c3acc(M, c3mul(U, acc), 1.0);
  } else {
    c3acc(M, c3mul(acc, U), -1.0);  // -S U^+  (C[p] = U^+)
  }
}

// one thread per link (site s, direction mu)
__global__ void force_kernel(Geom g, const double2* __restrict__ U, FieldPtr xf, FieldPtr yf,
                             const double2* __restrict__ W, double csw, double* __restrict__ F) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.V * 4) return;
  const long long s = t >> 2;
  const int mu = (int)(t & 3);
  const int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  int x[4];
  global_coords(g, blk, r, x);
  const C3 Ux = link64(g, U, s, mu);

  // ---- hopping part
  const long long sp = shifted(g, x, mu, 1, -1, 0);
  const int bp = (int)(sp / g.Vb), rp = (int)(sp - (long long)bp * g.Vb);
  const int xmu = mu == 0 ? x[0] : (mu == 1 ? x[1] : (mu == 2 ? x[2] : x[3]));
  const int Lmu = mu == 0 ? g.L[0] : (mu == 1 ? g.L[1] : (mu == 2 ? g.L[2] : g.L[3]));
  const double bcmu = mu == 0 ? g.bc[0] : (mu == 1 ? g.bc[1] : (mu == 2 ? g.bc[2] : g.bc[3]));
  const double eta = (xmu == Lmu - 1) ? bcmu : 1.0;
  Spinor<double> x_here = load_spinor<P64, double>(xf, g.Vb, blk, r);
  Spinor<double> y_here = load_spinor<P64, double>(yf, g.Vb, blk, r);
  Spinor<double> x_up = load_spinor<P64, double>(xf, g.Vb, bp, rp);
  Spinor<double> y_up = load_spinor<P64, double>(yf, g.Vb, bp, rp);
  Half<double> h, k, h2, k2;
  switch (mu) {
    case 0: h = project<0, -1>(x_up); k = project<0, -1>(y_here); h2 = project<0, 1>(x_here); k2 = project<0, 1>(y_up); break;
    case 1: h = project<1, -1>(x_up); k = project<1, -1>(y_here); h2 = project<1, 1>(x_here); k2 = project<1, 1>(y_up); break;
    case 2: h = project<2, -1>(x_up); k = project<2, -1>(y_here); h2 = project<2, 1>(x_here); k2 = project<2, 1>(y_up); break;
    default: h = project<3, -1>(x_up); k = project<3, -1>(y_here); h2 = project<3, 1>(x_here); k2 = project<3, 1>(y_up); break;
  }
  C3 P1, P2;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      P1.m[a][b] = cmul(h.c[0][a], conjg(k.c[0][b])) + cmul(h.c[1][a], conjg(k.c[1][b]));
      P2.m[a][b] = cmul(h2.c[0][a], conjg(k2.c[0][b])) + cmul(h2.c[1][a], conjg(k2.c[1][b]));
    }
  C3 Mh = c3mul(Ux, P1);
  c3acc(Mh, c3mul(P2, c3dag(Ux)), -1.0);
  cd th[8];
  trace_lambda(Mh, th);
  double out[8];
  for (int a = 0; a < 8; ++a) out[a] = -0.25 * eta * th[a].im;

  // ---- clover part
  if (csw != 0.0) {
    C3 Mc;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Mc.m[i][j] = {0, 0};
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == mu) continue;
      const int pl = plane(mu, nu);
      const long long s_mu = sp;                                // x + mu
      const long long s_nu = shifted(g, x, nu, 1, -1, 0);       // x + nu
      const long long s_mn = shifted(g, x, mu, 1, nu, 1);       // x + mu + nu
      const long long s_dn = shifted(g, x, nu, -1, -1, 0);      // x - nu
      const long long s_mdn = shifted(g, x, mu, 1, nu, -1);     // x + mu - nu
      C3 C[4];
      long long c[4];
      if (mu < nu) {
        // (mu, nu) orientation.  Plaquette at x: [U_mu(x), U_nu(x+mu), U_mu(x+nu)^+, U_nu(x)^+]
        C[0] = Ux; C[1] = link64(g, U, s_mu, nu); C[2] = c3dag(link64(g, U, s_nu, mu)); C[3] = c3dag(link64(g, U, s, nu));
        c[0] = s; c[1] = s_mu; c[2] = s_mn; c[3] = s_nu;
        plaquette_terms(C, c, 0, false, pl, W, Mc);
        // plaquette at x - nu: [U_mu(x-nu), U_nu(x+mu-nu), U_mu(x)^+, U_nu(x-nu)^+]
        C[0] = link64(g, U, s_dn, mu); C[1] = link64(g, U, s_mdn, nu); C[2] = c3dag(Ux); C[3] = c3dag(link64(g, U, s_dn, nu));
        c[0] = s_dn; c[1] = s_mdn; c[2] = s_mu; c[3] = s;
        plaquette_terms(C, c, 2, true, pl, W, Mc);
      } else {
        // (nu, mu) orientation.  Plaquette at x: [U_nu(x), U_mu(x+nu), U_nu(x+mu)^+, U_mu(x)^+]
        C[0] = link64(g, U, s, nu); C[1] = link64(g, U, s_nu, mu); C[2] = c3dag(link64(g, U, s_mu, nu)); C[3] = c3dag(Ux);
        c[0] = s; c[1] = s_nu; c[2] = s_mn; c[3] = s_mu;
        plaquette_terms(C, c, 3, true, pl, W, Mc);
        // plaquette at x - nu: [U_nu(x-nu), U_mu(x), U_nu(x+mu-nu)^+, U_mu(x-nu)^+]
        C[0] = link64(g, U, s_dn, nu); C[1] = Ux; C[2] = c3dag(link64(g, U, s_mdn, nu)); C[3] = c3dag(link64(g, U, s_dn, mu));
        c[0] = s_dn; c[1] = s; c[2] = s_mu; c[3] = s_mdn;
        plaquette_terms(C, c, 1, false, pl, W, Mc);
      }
    }
    cd tc[8];
    trace_lambda(Mc, tc);
    for (int a = 0; a < 8; ++a) out[a] += (csw / 32.0) * tc[a].re;
  }
  const long long lex = lex_index(g, x);
  for (int a = 0; a < 8; ++a) F[(lex * 4 + mu) * 8 + a] = out[a];
}

int force_apply(qcd_ctx* c, const Rec& x, const Rec& y, double* F, cudaStream_t s) {
  if (x.prec != P64 || y.prec != P64) return QCD_ERR_ARG;
  QCD_TRY(ensure_gauge(c, P64, s));
  double2* W = nullptr;
  const size_t wbytes = (size_t)c->V * 6 * 9 * sizeof(double2);
  if (cudaMalloc(&W, wbytes) != cudaSuccess) {
    cudaGetLastError();
    return QCD_ERR_NOMEM;
  }
  force_w_kernel<<<(unsigned)((c->V + 127) / 128), 128, 0, s>>>(c->g, x.ptr(), y.ptr(), W);
  int st = QCD_OK;
  {
    cudaError_t e = cudaGetLastError();
    g_launches.fetch_add(1);
    if (e != cudaSuccess) st = cuda_fail(e, "force_w_kernel");
  }
  if (st == QCD_OK) {
    force_kernel<<<(unsigned)((c->V * 4 + 127) / 128), 128, 0, s>>>(c->g, (const double2*)c->U[P64], x.ptr(),
                                                                     y.ptr(), W, c->p.csw, F);
    cudaError_t e = cudaGetLastError();
    g_launches.fetch_add(1);
    if (e != cudaSuccess) st = cuda_fail(e, "force_kernel");
  }
  cudaStreamSynchronize(s);
  cudaFree(W);
  return st;
}

}  // namespace qcd
