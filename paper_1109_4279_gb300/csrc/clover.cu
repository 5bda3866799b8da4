// Clover term (abstract / Sec. 1: "Wilson-Dirac solver with Clover term"):
// A(x) = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_{mu nu} Fhat_{mu nu}(x),
// built once per gauge field in FP64, plus the inverse of its two 6x6 chiral
// blocks on odd sites for the even/odd block solver (Sec. 5, Table 1).
#include "internal.h"

namespace qcd {

typedef cpx<double> cd;

struct M3 {
  cd m[3][3];
};

__device__ __forceinline__ M3 m3mul(const M3& a, const M3& b) {
  M3 r;
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

__device__ __forceinline__ M3 m3dag(const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[i][j] = conjg(a.m[j][i]);
  return r;
}

// link U_mu at global coordinates x + shift (periodic), from the FP64 copy
__device__ __forceinline__ M3 link_at(const Geom& g, const double2* U64, const int x[4], int mu, int s0, int s1,
                                      int d0, int d1) {
  int y[4];  // selects only, no dynamically indexed writes
#pragma unroll
  for (int d = 0; d < 4; ++d) y[d] = (x[d] + (d == d0 ? s0 : 0) + (d == d1 ? s1 : 0) + g.L[d]) % g.L[d];
  long long s = internal_index(g, y);
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  SU3<double> u = load_link<P64, double>(U64, g.Vb, blk, r, mu);
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) o.m[i][j] = u.m[i][j];
  return o;
}

// Fhat_{mu nu}(x) = (Q - Q^+) / 8, Q = sum of the four counter-clockwise leaves at x
__device__ M3 fhat(const Geom& g, const double2* U64, const int x[4], int mu, int nu) {
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
  M3 q = m3mul(m3mul(link_at(g, U64, x, mu, 0, 0, mu, nu), link_at(g, U64, x, nu, 1, 0, mu, nu)),
               m3mul(m3dag(link_at(g, U64, x, mu, 0, 1, mu, nu)), m3dag(link_at(g, U64, x, nu, 0, 0, mu, nu))));
  // leaf 2: U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
  M3 l = m3mul(m3mul(link_at(g, U64, x, nu, 0, 0, mu, nu), m3dag(link_at(g, U64, x, mu, -1, 1, mu, nu))),
               m3mul(m3dag(link_at(g, U64, x, nu, -1, 0, mu, nu)), link_at(g, U64, x, mu, -1, 0, mu, nu)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + l.m[i][j];
  // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
  l = m3mul(m3mul(m3dag(link_at(g, U64, x, mu, -1, 0, mu, nu)), m3dag(link_at(g, U64, x, nu, -1, -1, mu, nu))),
            m3mul(link_at(g, U64, x, mu, -1, -1, mu, nu), link_at(g, U64, x, nu, 0, -1, mu, nu)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + l.m[i][j];
  // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
  l = m3mul(m3mul(m3dag(link_at(g, U64, x, nu, 0, -1, mu, nu)), link_at(g, U64, x, mu, 0, -1, mu, nu)),
            m3mul(link_at(g, U64, x, nu, 1, -1, mu, nu), m3dag(link_at(g, U64, x, mu, 0, 0, mu, nu))));
  M3 f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd qij = q.m[i][j] + l.m[i][j];
      f.m[i][j] = qij;
    }
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) o.m[i][j] = 0.125 * (f.m[i][j] - conjg(f.m[j][i]));
  return o;
}

// pack the Hermitian 6x6 M into 36 reals: 6 diagonal, then (i < j) pairs row-major
__device__ __forceinline__ void pack_herm(const cd M[6][6], double* out) {
  for (int i = 0; i < 6; ++i) out[i] = M[i][i].re;
  int k = 6;
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      out[k++] = M[i][j].re;
      out[k++] = M[i][j].im;
    }
}

// Gauss-Jordan inverse with partial pivoting; returns false if singular
__device__ bool invert6(cd M[6][6], cd Inv[6][6]) {
  double scale = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      Inv[i][j] = {i == j ? 1.0 : 0.0, 0.0};
      scale = fmax(scale, fabs(M[i][j].re) + fabs(M[i][j].im));
    }
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    double best = 0;
    for (int r = col; r < 6; ++r) {
      double a = fabs(M[r][col].re) + fabs(M[r][col].im);
      if (a > best) {
        best = a;
        piv = r;
      }
    }
    if (!(best > 1e-14 * scale)) return false;
    if (piv != col)
      for (int j = 0; j < 6; ++j) {
        cd t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t;
        t = Inv[col][j]; Inv[col][j] = Inv[piv][j]; Inv[piv][j] = t;
      }
    cd d = M[col][col];
    double den = d.re * d.re + d.im * d.im;
    cd dinv = {d.re / den, -d.im / den};
    for (int j = 0; j < 6; ++j) {
      M[col][j] = cmul(M[col][j], dinv);
      Inv[col][j] = cmul(Inv[col][j], dinv);
    }
    for (int r = 0; r < 6; ++r) {
      if (r == col) continue;
      cd f = M[r][col];
      for (int j = 0; j < 6; ++j) {
        M[r][j] = M[r][j] - cmul(f, M[col][j]);
        Inv[r][j] = Inv[r][j] - cmul(f, Inv[col][j]);
      }
    }
  }
  return true;
}

__global__ void clover_build_kernel(Geom g, const double2* __restrict__ U64, double m0, double csw, FieldPtr A,
                                    FieldPtr Ahat, int* bad) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  int x[4];
  global_coords(g, blk, r, x);
  M3 F01 = fhat(g, U64, x, 0, 1), F02 = fhat(g, U64, x, 0, 2), F03 = fhat(g, U64, x, 0, 3);
  M3 F12 = fhat(g, U64, x, 1, 2), F13 = fhat(g, U64, x, 1, 3), F23 = fhat(g, U64, x, 2, 3);
  // sigma_0k = diag(s_k, -s_k); sigma_jk = -eps_jkl diag(s_l, s_l).  Hence
  // upper block: (i c/2) sum_k s_k (x) E_k, E = (F01 - F23, F02 + F13, F03 - F12);
  // lower block: -(i c/2) sum_k s_k (x) B_k, B = (F01 + F23, F02 - F13, F03 + F12).
  double rec[72], inv[72];
  const bool odd = r >= g.Vbh;
  for (int chir = 0; chir < 2; ++chir) {
    const double sg = chir == 0 ? 1.0 : -1.0;
    cd M[6][6];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        cd E1 = F01.m[a][b] - sg * F23.m[a][b];
        cd E2 = F02.m[a][b] + sg * F13.m[a][b];
        cd E3 = F03.m[a][b] - sg * F12.m[a][b];
        // s1 E1 + s2 E2 + s3 E3 = [[E3, E1 - i E2], [E1 + i E2, -E3]]
        cd b00 = E3, b01 = E1 - ti(E2), b10 = E1 + ti(E2), b11 = -E3;
        const double f = 0.5 * csw * sg;
        M[a][b] = f * ti(b00);
        M[a][3 + b] = f * ti(b01);
        M[3 + a][b] = f * ti(b10);
        M[3 + a][3 + b] = f * ti(b11);
      }
    for (int i = 0; i < 6; ++i) M[i][i].re += 4.0 + m0;
    pack_herm(M, rec + 36 * chir);
    if (odd) {
      cd Inv[6][6];
      if (!invert6(M, Inv)) atomicExch(bad, 1);
      // symmetrise the inverse (Hermitian up to rounding)
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
          cd a = Inv[i][j], b = conjg(Inv[j][i]);
          Inv[i][j] = 0.5 * (a + b);
          Inv[j][i] = conjg(Inv[i][j]);
        }
      pack_herm(Inv, inv + 36 * chir);
    }
  }
  store_record<P64, 72, double>(A, g.Vb, blk, r, rec);
  store_record<P64, 72, double>(Ahat, g.Vb, blk, r, odd ? inv : rec);
}

int build_clover(qcd_ctx* c, cudaStream_t s) {
  if (!c->gauge_loaded) return QCD_ERR_STATE;
  ++c->gen;  // every clover record is reallocated
  for (int p = 0; p < 5; ++p) {
    rec_free(c->A[p]);
    rec_free(c->Ahat[p]);
  }
  QCD_TRY(rec_alloc(c->A[P64], P64, 72, c->V));
  QCD_TRY(rec_alloc(c->Ahat[P64], P64, 72, c->V));
  int* d_bad = (int*)c->d_scalars;
  QCD_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
  clover_build_kernel<<<(unsigned)((c->V + 127) / 128), 128, 0, s>>>(
      c->g, (const double2*)c->U[P64], c->p.m0, c->p.csw, c->A[P64].ptr(), c->Ahat[P64].ptr(), d_bad);
  QCD_LAUNCHED();
  int h = 0;
  QCD_CUDA(cudaMemcpyAsync(&h, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  if (h) return QCD_ERR_SINGULAR_CLOVER;
  c->clover_built = true;
  return QCD_OK;
}

int ensure_clover(qcd_ctx* c, int prec, cudaStream_t s) {
  if (!c->clover_built) return QCD_ERR_STATE;
  if (c->A[prec].data) return QCD_OK;
  ++c->gen;
  QCD_TRY(rec_alloc(c->A[prec], prec, 72, c->V));
  QCD_TRY(rec_alloc(c->Ahat[prec], prec, 72, c->V));
  QCD_TRY(convert_rec(c, c->A[P64], c->A[prec], s));
  QCD_TRY(convert_rec(c, c->Ahat[P64], c->Ahat[prec], s));
  return QCD_OK;
}

}  // namespace qcd
