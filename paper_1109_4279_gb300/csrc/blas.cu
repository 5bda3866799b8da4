// FP64 spinor linear algebra of the FGCR recursion (Sec. 4; Sec. 6 counts it
// as "spinor linear algebra", 12 % of the solver time on QPACE): fused
// multi-dot / multi-axpy kernels for classical Gram-Schmidt with
// re-orthogonalisation, norms and the solution update.  Every reduction is
// deterministic: fixed grid, per-CTA partial sums in a fixed order, then one
// CTA sums the partials in index order.
#include "internal.h"

namespace qcd {

static constexpr int kMaxVec = 64;
static constexpr int kBlasThreads = 256;

struct VecList {
  const double2* v[kMaxVec];
};

static unsigned blas_grid(long long n) {
  long long g = (n + kBlasThreads - 1) / kBlasThreads;
  const long long cap = 152 * 8;  // a few CTAs per SM; grid-stride beyond
  return (unsigned)(g < cap ? (g < 1 ? 1 : g) : cap);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// reduce M values per thread over the CTA; thread 0 writes part[blockIdx.x * M + j]
template <int M>
__device__ __forceinline__ void cta_reduce_store(double (&v)[M], double* part) {
  __shared__ double sh[kBlasThreads / 32][M > 0 ? M : 1];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double t = warp_sum(v[j]);
    if (l == 0) sh[w][j] = t;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double t = 0;
    for (int k = 0; k < kBlasThreads / 32; ++k) t += sh[k][threadIdx.x];
    part[(long long)blockIdx.x * M + threadIdx.x] = t;
  }
}

__global__ void reduce_partials_kernel(const double* __restrict__ part, int nparts, int stride, int m, double* out) {
  // one warp per value, lanes stride over partials in a fixed order
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int l = threadIdx.x & 31;
  if (j >= m) return;
  double t = 0;
  for (int p = l; p < nparts; p += 32) t += part[(long long)p * stride + j];
  t = warp_sum(t);
  if (l == 0) out[j] = t;
}

// out[j] = sum_p partials[p * stride + j], j < m
int reduce_partials(const double* partials, int nparts, int stride, int m, double* out, cudaStream_t s) {
  const int warps = 8;
  reduce_partials_kernel<<<(m + warps - 1) / warps, 32 * warps, 0, s>>>(partials, nparts, stride, m, out);
  QCD_LAUNCHED();
  return QCD_OK;
}

// true if the Gram-Schmidt pass must be repeated (DGKS criterion): the first
// pass left less than half of the squared norm, |chi'|^2 < |chi|^2 / 2.
// gs = {|chi|^2, |chi'|^2, ...}; a null gs means "always".
__device__ __forceinline__ bool second_pass_needed(const double* gs) {
  return gs == nullptr || gs[1] < 0.5 * gs[0];
}

// out[j] = (v_j, w) = sum conj(v_j) w, j < k <= K; with NORM also out[2K] = |w|^2.
// cond (optional): skip unless second_pass_needed(cond) -- then the partial
// sums are zero, so the reduced coefficients are zero.
template <int K, int NORM>
__global__ void __launch_bounds__(kBlasThreads) multidot_kernel(VecList vl, int k, const double2* __restrict__ w,
                                                                long long n, const double* cond, double* part) {
  double acc[2 * K + NORM];
#pragma unroll
  for (int j = 0; j < 2 * K + NORM; ++j) acc[j] = 0;
  if (cond == nullptr || second_pass_needed(cond)) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const double2 b = __ldg(w + i);
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < k) {
          const double2 a = __ldg(vl.v[j] + i);
          acc[2 * j] = fma(a.x, b.x, fma(a.y, b.y, acc[2 * j]));
          acc[2 * j + 1] = fma(a.x, b.y, fma(-a.y, b.x, acc[2 * j + 1]));
        }
      if (NORM) acc[2 * K] = fma(b.x, b.x, fma(b.y, b.y, acc[2 * K]));
    }
  }
  cta_reduce_store<2 * K + NORM>(acc, part);
}

// w -= sum_j c_j v_j; then out[j] = (v_j, w) (DOT = 1) or out = {|w|^2, (w, rho)} (DOT = 2)
template <int K, int DOT>
__global__ void __launch_bounds__(kBlasThreads) axpy_dot_kernel(VecList vl, int k, const double* __restrict__ coef,
                                                                double2* __restrict__ w,
                                                                const double2* __restrict__ rho, long long n,
                                                                const double* cond, double* part) {
  constexpr int M = DOT == 1 ? 2 * K : 3;
  if (cond != nullptr && !second_pass_needed(cond)) return;  // block-uniform: no partials written
  double acc[M];
#pragma unroll
  for (int j = 0; j < M; ++j) acc[j] = 0;
  double2 cf[K];
#pragma unroll
  for (int j = 0; j < K; ++j) cf[j] = j < k ? make_double2(coef[2 * j], coef[2 * j + 1]) : make_double2(0, 0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 b = w[i];
    double2 a[K];
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) {
        a[j] = __ldg(vl.v[j] + i);
        b.x -= cf[j].x * a[j].x - cf[j].y * a[j].y;
        b.y -= cf[j].x * a[j].y + cf[j].y * a[j].x;
      }
    w[i] = b;
    if (DOT == 1) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < k) {
          acc[2 * j] = fma(a[j].x, b.x, fma(a[j].y, b.y, acc[2 * j]));
          acc[2 * j + 1] = fma(a[j].x, b.y, fma(-a[j].y, b.x, acc[2 * j + 1]));
        }
    } else {
      const double2 r = __ldg(rho + i);
      acc[0] = fma(b.x, b.x, fma(b.y, b.y, acc[0]));
      acc[1] = fma(b.x, r.x, fma(b.y, r.y, acc[1]));
      acc[2] = fma(b.x, r.y, fma(-b.y, r.x, acc[2]));
    }
  }
  cta_reduce_store<M>(acc, part);
}

// Final Gram-Schmidt coefficients of iteration k: gs = {|chi|^2 before,
// pass-1 {|chi'|^2, Re, Im (chi', rho)}, pass-2 {...}}; the pass-2 values
// are used when the second pass ran.  Thread 0 of CTA 0 stores them in
// cr = {|chi_k|^2, (chi_k, rho_k)}.  Then chi /= |chi|;
// rho -= ((chi, rho) / |chi|^2) chi_unnormalised;  partial |rho|^2.
__global__ void __launch_bounds__(kBlasThreads) normalise_update_kernel(double2* __restrict__ chi,
                                                                        double2* __restrict__ rho,
                                                                        const double* __restrict__ gs, int two_pass,
                                                                        double* cr, long long n, double* part) {
  const double* co = (two_pass && second_pass_needed(gs)) ? gs + 4 : gs + 1;
  const double nrm2 = co[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cr[0] = co[0];
    cr[1] = co[1];
    cr[2] = co[2];
  }
  const double inv = nrm2 > 0 ? 1.0 / sqrt(nrm2) : 0.0;
  const double cre = nrm2 > 0 ? co[1] / nrm2 : 0.0, cim = nrm2 > 0 ? co[2] / nrm2 : 0.0;
  double acc[1] = {0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 x = chi[i];
    double2 r = rho[i];
    r.x -= cre * x.x - cim * x.y;
    r.y -= cre * x.y + cim * x.x;
    rho[i] = r;
    chi[i] = make_double2(x.x * inv, x.y * inv);
    acc[0] = fma(r.x, r.x, fma(r.y, r.y, acc[0]));
  }
  cta_reduce_store<1>(acc, part);
}

// x += sum_j g_j phi_j
template <int K>
__global__ void __launch_bounds__(kBlasThreads) multi_axpy_kernel(VecList vl, int k, const double* __restrict__ gam,
                                                                  double2* __restrict__ x, long long n) {
  double2 cf[K];
#pragma unroll
  for (int j = 0; j < K; ++j) cf[j] = j < k ? make_double2(gam[2 * j], gam[2 * j + 1]) : make_double2(0, 0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 b = x[i];
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) {
        const double2 a = __ldg(vl.v[j] + i);
        b.x += cf[j].x * a.x - cf[j].y * a.y;
        b.y += cf[j].x * a.y + cf[j].y * a.x;
      }
    x[i] = b;
  }
}

__global__ void __launch_bounds__(kBlasThreads) norm2_kernel(const double2* __restrict__ v, long long n, double* part) {
  double acc[1] = {0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 a = __ldg(v + i);
    acc[0] = fma(a.x, a.x, fma(a.y, a.y, acc[0]));
  }
  cta_reduce_store<1>(acc, part);
}

// y = g5 x on the internal FP64 layout [blk][12 components][Vb]: components 6..11 are spins 2, 3
__global__ void gamma5_kernel(const double2* __restrict__ x, double2* __restrict__ y, int Vb, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int comp = (int)((i / Vb) % 12);
    double2 a = x[i];
    if (comp >= 6) a = make_double2(-a.x, -a.y);
    y[i] = a;
  }
}

// FGCR back substitution (one thread): H gamma = c with H upper triangular,
// H_kk = |chi_k| after Gram-Schmidt, H_jk = a1_jk + a2_jk (j < k, the two
// classical Gram-Schmidt passes of iteration k), c_k = (chi_k, rho_k) / H_kk.
// a1, a2: complex, iteration k's coefficients at (k * ld + j); cr: per k
// {|chi_k|^2, Re (chi_k, rho_k), Im (chi_k, rho_k)}; gam: out, complex.
__global__ void backsub_kernel(const double* a1, const double* a2, const double* cr, int k, int ld, double* gam) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    const double hkk = sqrt(cr[3 * i]);
    double sr = cr[3 * i + 1] / hkk, si = cr[3 * i + 2] / hkk;
    for (int j = i + 1; j < k; ++j) {
      const long long o = ((long long)j * ld + i) * 2;  // H_ij is computed in iteration j
      const double hr = a1[o] + a2[o], hi = a1[o + 1] + a2[o + 1];
      const double gr = gam[2 * j], gi = gam[2 * j + 1];
      sr -= hr * gr - hi * gi;
      si -= hr * gi + hi * gr;
    }
    gam[2 * i] = sr / hkk;
    gam[2 * i + 1] = si / hkk;
  }
}

// ------------------------------------------------------------------------
static VecList make_list(const double* const* v, int k) {
  VecList vl;
  for (int j = 0; j < kMaxVec; ++j) vl.v[j] = j < k ? (const double2*)v[j] : nullptr;
  return vl;
}

int blas_multidot(qcd_ctx* c, double* part, const double* const* v, int k, const double* w, double* d_out, cudaStream_t s,
                  const double* cond, double* d_norm) {
  if (k <= 0) return QCD_OK;
  if (k > kMaxVec) return QCD_ERR_ARG;
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 16.0 * n * (k + 1), 8.0 * n * k);
  int K;
  if (k <= 4) K = 4; else if (k <= 8) K = 8; else if (k <= 16) K = 16; else K = 32;
  int done = 0;
  while (done < k) {
    const int kk = k - done < K ? k - done : K;
    const int norm = (d_norm != nullptr && done == 0) ? 1 : 0;
    const int M = 2 * K + norm;
    VecList vl = make_list(v + done, kk);
    const double2* w2 = (const double2*)w;
#define MD(KK)                                                                                                   \
  if (norm)                                                                                                      \
    multidot_kernel<KK, 1><<<grid, kBlasThreads, 0, s>>>(vl, kk, w2, n, cond, part);                  \
  else                                                                                                           \
    multidot_kernel<KK, 0><<<grid, kBlasThreads, 0, s>>>(vl, kk, w2, n, cond, part);
    switch (K) {
      case 4: MD(4); break;
      case 8: MD(8); break;
      case 16: MD(16); break;
      default: MD(32); break;
    }
#undef MD
    QCD_LAUNCHED();
    QCD_TRY(reduce_partials(part, (int)grid, M, 2 * kk, d_out + 2 * done, s));
    if (norm) QCD_TRY(reduce_partials(part + 2 * K, (int)grid, M, 1, d_norm, s));
    done += kk;
  }
  return QCD_OK;
}

template <int DOT>
static int axpy_dot_impl(qcd_ctx* c, double* part, const double* const* v, int k, const double* d_coef, double* w, const double* rho,
                         double* d_out, cudaStream_t s, const double* cond = nullptr) {
  if (k > 32) return QCD_ERR_UNSUPPORTED;
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  int K;
  if (k <= 4) K = 4; else if (k <= 8) K = 8; else if (k <= 16) K = 16; else K = 32;
  const int M = DOT == 1 ? 2 * K : 3;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 16.0 * n * (k + 2 + (DOT == 2)), 16.0 * n * k);
  VecList vl = make_list(v, k);
  const double2* r2 = (const double2*)rho;
  switch (K) {
    case 4: axpy_dot_kernel<4, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, (double2*)w, r2, n, cond, part); break;
    case 8: axpy_dot_kernel<8, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, (double2*)w, r2, n, cond, part); break;
    case 16: axpy_dot_kernel<16, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, (double2*)w, r2, n, cond, part); break;
    default: axpy_dot_kernel<32, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, (double2*)w, r2, n, cond, part); break;
  }
  QCD_LAUNCHED();
  return reduce_partials(part, (int)grid, M, DOT == 1 ? 2 * k : 3, d_out, s);
}

int blas_axpy_dot(qcd_ctx* c, double* part, const double* const* v, int k, const double* d_coef, double* w, double* d_out,
                  cudaStream_t s) {
  if (k <= 0) return QCD_OK;
  return axpy_dot_impl<1>(c, part, v, k, d_coef, w, nullptr, d_out, s);
}

int blas_axpy_norm_dot(qcd_ctx* c, double* part, const double* const* v, int k, const double* d_coef, double* w, const double* rho,
                       double* d_out, cudaStream_t s, const double* cond) {
  if (k <= 0) {
    // nothing to subtract: only the norm and the dot
    const long long n = c->V * 12;
    const unsigned grid = blas_grid(n);
    VecList vl = make_list(v, 0);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 32.0 * n, 8.0 * n);
    axpy_dot_kernel<4, 2><<<grid, kBlasThreads, 0, s>>>(vl, 0, d_coef, (double2*)w, (const double2*)rho, n, cond,
                                                        part);
    QCD_LAUNCHED();
    return reduce_partials(part, (int)grid, 3, 3, d_out, s);
  }
  return axpy_dot_impl<2>(c, part, v, k, d_coef, w, rho, d_out, s, cond);
}

int blas_normalise_update(qcd_ctx* c, double* part, double* chi, double* rho, const double* d_gs, int two_pass, double* d_cr,
                          double* d_out, cudaStream_t s) {
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 64.0 * n, 8.0 * n);
    normalise_update_kernel<<<grid, kBlasThreads, 0, s>>>((double2*)chi, (double2*)rho, d_gs, two_pass, d_cr, n,
                                                          part);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_out, s);
}

int blas_multi_axpy(qcd_ctx* c, const double* const* phi, int k, const double* d_gamma, double* x, cudaStream_t s) {
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  int done = 0;
  while (done < k) {
    int kk = k - done < 16 ? k - done : 16;
    VecList vl = make_list(phi + done, kk);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 16.0 * n * (kk + 2), 8.0 * n * kk);
    if (kk <= 4)
      multi_axpy_kernel<4><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, n);
    else if (kk <= 8)
      multi_axpy_kernel<8><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, n);
    else
      multi_axpy_kernel<16><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, n);
    QCD_LAUNCHED();
    done += kk;
  }
  return QCD_OK;
}

int blas_norm2(qcd_ctx* c, double* part, const double* v, double* d_out, cudaStream_t s) {
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 16.0 * n, 4.0 * n);
    norm2_kernel<<<grid, kBlasThreads, 0, s>>>((const double2*)v, n, part);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_out, s);
}

int blas_gamma5(qcd_ctx* c, const double* x, double* y, int, cudaStream_t s) {
  const long long n = c->V * 12;
  gamma5_kernel<<<blas_grid(n), kBlasThreads, 0, s>>>((const double2*)x, (double2*)y, c->g.Vb, n);
  QCD_LAUNCHED();
  return QCD_OK;
}

int fgcr_backsub(const double* d_a1, const double* d_a2, const double* d_cr, int k, int ld, double* d_gamma,
                 cudaStream_t s) {
  backsub_kernel<<<1, 32, 0, s>>>(d_a1, d_a2, d_cr, k, ld, d_gamma);
  QCD_LAUNCHED();
  return QCD_OK;
}

}  // namespace qcd
