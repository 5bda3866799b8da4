// Spinor linear algebra of the FGCR recursion (Sec. 4; Sec. 6 counts it as
// "spinor linear algebra", 12 % of the solver time on QPACE): fused
// multi-dot / multi-axpy kernels for classical Gram-Schmidt with
// re-orthogonalisation, norms and the solution update, in FP64 (vectors of
// double2, one complex number per element) or FP32 (vectors of float4, two
// complex numbers per element; the recursion of the mixed-precision scheme).
// FP32 kernels accumulate in FP32 per thread; every CTA and grid sum is FP64.
// Every reduction is deterministic: fixed grid, per-CTA partial sums in a
// fixed order, then one warp per value sums the partials in index order.
#include "internal.h"

namespace qcd {

static constexpr int kMaxVec = 64;
static constexpr int kBlasThreads = 256;

template <typename R>
struct VecT;
template <>
struct VecT<double> {
  typedef double2 type;
  static constexpr int NC = 1;  // complex numbers per element
};
template <>
struct VecT<float> {
  typedef float4 type;
  static constexpr int NC = 2;
};

template <typename E>
struct VecList {
  const E* v[kMaxVec];
};

// ---- complex arithmetic on one element
// (re, im) += conj(a) b
__device__ __forceinline__ void dot_acc(const double2& a, const double2& b, double& re, double& im) {
  re = fma(a.x, b.x, fma(a.y, b.y, re));
  im = fma(a.x, b.y, fma(-a.y, b.x, im));
}
__device__ __forceinline__ void dot_acc(const float4& a, const float4& b, float& re, float& im) {
  re = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, re))));
  im = fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, fmaf(-a.w, b.z, im))));
}
__device__ __forceinline__ void nrm_acc(const double2& b, double& n) { n = fma(b.x, b.x, fma(b.y, b.y, n)); }
__device__ __forceinline__ void nrm_acc(const float4& b, float& n) {
  n = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, n))));
}
// b -= (cr + i ci) a, two fused multiply-adds per real (the FP64 pipe is the
// bound of these kernels on GB300)
__device__ __forceinline__ void csub(double2& b, double cr, double ci, const double2& a) {
  b.x = fma(-cr, a.x, fma(ci, a.y, b.x));
  b.y = fma(-cr, a.y, fma(-ci, a.x, b.y));
}
__device__ __forceinline__ void csub(float4& b, float cr, float ci, const float4& a) {
  b.x = fmaf(-cr, a.x, fmaf(ci, a.y, b.x));
  b.y = fmaf(-cr, a.y, fmaf(-ci, a.x, b.y));
  b.z = fmaf(-cr, a.z, fmaf(ci, a.w, b.z));
  b.w = fmaf(-cr, a.w, fmaf(-ci, a.z, b.w));
}
// b += (cr + i ci) a
__device__ __forceinline__ void cadd(double2& b, double cr, double ci, const double2& a) {
  b.x = fma(cr, a.x, fma(-ci, a.y, b.x));
  b.y = fma(cr, a.y, fma(ci, a.x, b.y));
}
__device__ __forceinline__ void cadd(float4& b, float cr, float ci, const float4& a) {
  b.x = fmaf(cr, a.x, fmaf(-ci, a.y, b.x));
  b.y = fmaf(cr, a.y, fmaf(ci, a.x, b.y));
  b.z = fmaf(cr, a.z, fmaf(-ci, a.w, b.z));
  b.w = fmaf(cr, a.w, fmaf(ci, a.z, b.w));
}
__device__ __forceinline__ double2 rscale(const double2& a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float4 rscale(const float4& a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}

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

// reduce M values per thread over the CTA (in FP64); thread j < M writes
// part[blockIdx.x * M + j]
template <int M, typename A>
__device__ __forceinline__ void cta_reduce_store(A (&v)[M], double* part) {
  __shared__ double sh[kBlasThreads / 32][M > 0 ? M : 1];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double t = warp_sum((double)v[j]);
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
template <typename R, int K, int NORM>
__global__ void __launch_bounds__(kBlasThreads)
    multidot_kernel(VecList<typename VecT<R>::type> vl, int k, const typename VecT<R>::type* __restrict__ w, long long n,
                    const double* cond, double* part) {
  typedef typename VecT<R>::type E;
  R acc[2 * K + NORM];
#pragma unroll
  for (int j = 0; j < 2 * K + NORM; ++j) acc[j] = 0;
  if (cond == nullptr || second_pass_needed(cond)) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const E b = __ldg(w + i);
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < k) dot_acc(__ldg(vl.v[j] + i), b, acc[2 * j], acc[2 * j + 1]);
      if (NORM) nrm_acc(b, acc[2 * K]);
    }
  }
  cta_reduce_store<2 * K + NORM>(acc, part);
}

// w -= sum_j c_j v_j; then out[j] = (v_j, w) (DOT = 1) or out = {|w|^2, (w, rho)} (DOT = 2)
template <typename R, int K, int DOT>
__global__ void __launch_bounds__(kBlasThreads)
    axpy_dot_kernel(VecList<typename VecT<R>::type> vl, int k, const double* __restrict__ coef,
                    typename VecT<R>::type* __restrict__ w, const typename VecT<R>::type* __restrict__ rho, long long n,
                    const double* cond, double* part) {
  typedef typename VecT<R>::type E;
  constexpr int M = DOT == 1 ? 2 * K : 3;
  if (cond != nullptr && !second_pass_needed(cond)) return;  // block-uniform: no partials written
  R acc[M];
#pragma unroll
  for (int j = 0; j < M; ++j) acc[j] = 0;
  R cr[K], ci[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    cr[j] = j < k ? (R)coef[2 * j] : R(0);
    ci[j] = j < k ? (R)coef[2 * j + 1] : R(0);
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    E b = w[i];
    E a[K];
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) {
        a[j] = __ldg(vl.v[j] + i);
        csub(b, cr[j], ci[j], a[j]);
      }
    w[i] = b;
    if (DOT == 1) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < k) dot_acc(a[j], b, acc[2 * j], acc[2 * j + 1]);
    } else {
      const E r = __ldg(rho + i);
      nrm_acc(b, acc[0]);
      dot_acc(b, r, acc[1], acc[2]);
    }
  }
  cta_reduce_store<M>(acc, part);
}

// Final Gram-Schmidt coefficients of iteration k: gs = {|chi|^2 before,
// pass-1 {|chi'|^2, Re, Im (chi', rho)}, pass-2 {...}}; the pass-2 values
// are used when the second pass ran.  Thread 0 of CTA 0 stores them in
// cr = {|chi_k|^2, (chi_k, rho_k)}.  Then chi /= |chi|;
// rho -= ((chi, rho) / |chi|^2) chi_unnormalised;  partial |rho|^2.
template <typename R>
__global__ void __launch_bounds__(kBlasThreads)
    normalise_update_kernel(typename VecT<R>::type* __restrict__ chi, typename VecT<R>::type* __restrict__ rho,
                            const double* __restrict__ gs, int two_pass, double* cr, long long n, double* part) {
  typedef typename VecT<R>::type E;
  const double* co = (two_pass && second_pass_needed(gs)) ? gs + 4 : gs + 1;
  const double nrm2 = co[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cr[0] = co[0];
    cr[1] = co[1];
    cr[2] = co[2];
  }
  const R inv = nrm2 > 0 ? (R)(1.0 / sqrt(nrm2)) : R(0);
  const R cre = nrm2 > 0 ? (R)(co[1] / nrm2) : R(0), cim = nrm2 > 0 ? (R)(co[2] / nrm2) : R(0);
  R acc[1] = {0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const E x = chi[i];
    E r = rho[i];
    csub(r, cre, cim, x);
    rho[i] = r;
    chi[i] = rscale(x, inv);
    nrm_acc(r, acc[0]);
  }
  cta_reduce_store<1>(acc, part);
}

// x += sum_j g_j phi_j
template <typename R, int K>
__global__ void __launch_bounds__(kBlasThreads)
    multi_axpy_kernel(VecList<typename VecT<R>::type> vl, int k, const double* __restrict__ gam,
                      typename VecT<R>::type* __restrict__ x, long long n) {
  typedef typename VecT<R>::type E;
  R cr[K], ci[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    cr[j] = j < k ? (R)gam[2 * j] : R(0);
    ci[j] = j < k ? (R)gam[2 * j + 1] : R(0);
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    E b = x[i];
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) cadd(b, cr[j], ci[j], __ldg(vl.v[j] + i));
    x[i] = b;
  }
}

// Iterative refinement (Sec. 4): x64 += |r| sum_j g_j phi_j with FP32 phi_j,
// the sum formed in FP32 and added to the FP64 solution in FP64.  Element i
// of the FP32 layout [blk][6][Vb] (float4) holds the reals of FP64 elements
// (blk, 2c, r) and (blk, 2c + 1, r) of the layout [blk][12][Vb] (double2).
template <int K>
__global__ void __launch_bounds__(kBlasThreads)
    refine_update_kernel(VecList<float4> vl, int k, const double* __restrict__ gam, const double* __restrict__ rn2,
                         double2* __restrict__ x, int Vb, long long n) {
  float cr[K], ci[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    cr[j] = j < k ? (float)gam[2 * j] : 0.f;
    ci[j] = j < k ? (float)gam[2 * j + 1] : 0.f;
  }
  const double scale = sqrt(*rn2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float4 d = make_float4(0, 0, 0, 0);
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) cadd(d, cr[j], ci[j], __ldg(vl.v[j] + i));
    const long long blk = i / (6LL * Vb), rem = i - blk * 6LL * Vb;
    const long long c = rem / Vb, r = rem - c * Vb;
    const long long e0 = (blk * 12 + 2 * c) * Vb + r;
    double2 x0 = x[e0], x1 = x[e0 + Vb];
    x0.x = fma(scale, f32_to_f64(d.x), x0.x);  // widening on the integer pipes
    x0.y = fma(scale, f32_to_f64(d.y), x0.y);
    x1.x = fma(scale, f32_to_f64(d.z), x1.x);
    x1.y = fma(scale, f32_to_f64(d.w), x1.y);
    x[e0] = x0;
    x[e0 + Vb] = x1;
  }
}

// rho32 = r64 / |r|: the normalised FP64 residual as the FP32 source of a
// refinement cycle (same element mapping as refine_update_kernel)
__global__ void __launch_bounds__(kBlasThreads)
    demote_normalised_kernel(const double2* __restrict__ r, const double* __restrict__ rn2, float4* __restrict__ out,
                             int Vb, long long n) {
  const double inv = *rn2 > 0 ? 1.0 / sqrt(*rn2) : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long blk = i / (6LL * Vb), rem = i - blk * 6LL * Vb;
    const long long c = rem / Vb, rr = rem - c * Vb;
    const long long e0 = (blk * 12 + 2 * c) * Vb + rr;
    const double2 a = __ldg(r + e0), b = __ldg(r + e0 + Vb);
    out[i] = make_float4(f64_to_f32(a.x * inv), f64_to_f32(a.y * inv), f64_to_f32(b.x * inv), f64_to_f32(b.y * inv));
  }
}

template <typename R>
__global__ void __launch_bounds__(kBlasThreads)
    norm2_kernel(const typename VecT<R>::type* __restrict__ v, long long n, double* part) {
  R acc[1] = {0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    nrm_acc(__ldg(v + i), acc[0]);
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
template <typename R>
static VecList<typename VecT<R>::type> make_list(const R* const* v, int k) {
  VecList<typename VecT<R>::type> vl;
  for (int j = 0; j < kMaxVec; ++j) vl.v[j] = j < k ? (const typename VecT<R>::type*)v[j] : nullptr;
  return vl;
}

// elements of one 24-real-per-site field
template <typename R>
static long long nel(qcd_ctx* c) {
  return c->V * 12 / VecT<R>::NC;
}

static int pick_k(int k) { return k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 16 ? 16 : 32)); }

template <typename R>
int blas_multidot(qcd_ctx* c, double* part, const R* const* v, int k, const R* w, double* d_out, cudaStream_t s,
                  const double* cond, double* d_norm) {
  typedef typename VecT<R>::type E;
  if (k <= 0) return QCD_OK;
  if (k > kMaxVec) return QCD_ERR_ARG;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  // a conditional (second Gram-Schmidt) pass is counted as no work: the host
  // cannot know whether it runs, and on well-conditioned bases it returns at once
  const double work = cond ? 0.0 : 1.0;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, work * sizeof(E) * (double)n * (k + 1), work * 8.0 * c->V * 12 * k);
  const int K = pick_k(k);
  int done = 0;
  while (done < k) {
    const int kk = k - done < K ? k - done : K;
    const int norm = (d_norm != nullptr && done == 0) ? 1 : 0;
    const int M = 2 * K + norm;
    auto vl = make_list<R>(v + done, kk);
    const E* w2 = (const E*)w;
#define MD(KK)                                                                         \
  if (norm)                                                                            \
    multidot_kernel<R, KK, 1><<<grid, kBlasThreads, 0, s>>>(vl, kk, w2, n, cond, part); \
  else                                                                                 \
    multidot_kernel<R, KK, 0><<<grid, kBlasThreads, 0, s>>>(vl, kk, w2, n, cond, part);
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

template <typename R, int DOT>
static int axpy_dot_impl(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, const R* rho,
                         double* d_out, cudaStream_t s, const double* cond = nullptr) {
  typedef typename VecT<R>::type E;
  if (k > 32) return QCD_ERR_UNSUPPORTED;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  const int K = pick_k(k);
  const int M = DOT == 1 ? 2 * K : 3;
  const double work = cond ? 0.0 : 1.0;  // conditional pass: counted as no work (see blas_multidot)
  ProfScope ps(c, QCD_KERNEL_BLAS, s, work * sizeof(E) * (double)n * (k + 2 + (DOT == 2)),
               work * 16.0 * c->V * 12 * k);
  auto vl = make_list<R>(v, k);
  const E* r2 = (const E*)rho;
  E* w2 = (E*)w;
  switch (K) {
    case 4: axpy_dot_kernel<R, 4, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part); break;
    case 8: axpy_dot_kernel<R, 8, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part); break;
    case 16: axpy_dot_kernel<R, 16, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part); break;
    default: axpy_dot_kernel<R, 32, DOT><<<grid, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part); break;
  }
  QCD_LAUNCHED();
  return reduce_partials(part, (int)grid, M, DOT == 1 ? 2 * k : 3, d_out, s);
}

template <typename R>
int blas_axpy_dot(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, double* d_out,
                  cudaStream_t s) {
  if (k <= 0) return QCD_OK;
  return axpy_dot_impl<R, 1>(c, part, v, k, d_coef, w, nullptr, d_out, s);
}

template <typename R>
int blas_axpy_norm_dot(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, const R* rho,
                       double* d_out, cudaStream_t s, const double* cond) {
  typedef typename VecT<R>::type E;
  if (k <= 0) {
    // nothing to subtract: only the norm and the dot
    const long long n = nel<R>(c);
    const unsigned grid = blas_grid(n);
    auto vl = make_list<R>(v, 0);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 2.0 * sizeof(E) * n, 8.0 * c->V * 12);
    axpy_dot_kernel<R, 4, 2><<<grid, kBlasThreads, 0, s>>>(vl, 0, d_coef, (E*)w, (const E*)rho, n, cond, part);
    QCD_LAUNCHED();
    return reduce_partials(part, (int)grid, 3, 3, d_out, s);
  }
  return axpy_dot_impl<R, 2>(c, part, v, k, d_coef, w, rho, d_out, s, cond);
}

template <typename R>
int blas_normalise_update(qcd_ctx* c, double* part, R* chi, R* rho, const double* d_gs, int two_pass, double* d_cr,
                          double* d_out, cudaStream_t s) {
  typedef typename VecT<R>::type E;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 4.0 * sizeof(E) * n, 8.0 * c->V * 12);
    normalise_update_kernel<R><<<grid, kBlasThreads, 0, s>>>((E*)chi, (E*)rho, d_gs, two_pass, d_cr, n, part);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_out, s);
}

template <typename R>
int blas_multi_axpy(qcd_ctx* c, const R* const* phi, int k, const double* d_gamma, R* x, cudaStream_t s) {
  typedef typename VecT<R>::type E;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  int done = 0;
  while (done < k) {
    int kk = k - done < 16 ? k - done : 16;
    auto vl = make_list<R>(phi + done, kk);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, sizeof(E) * (double)n * (kk + 2), 8.0 * c->V * 12 * kk);
    if (kk <= 4)
      multi_axpy_kernel<R, 4><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (E*)x, n);
    else if (kk <= 8)
      multi_axpy_kernel<R, 8><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (E*)x, n);
    else
      multi_axpy_kernel<R, 16><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (E*)x, n);
    QCD_LAUNCHED();
    done += kk;
  }
  return QCD_OK;
}

int blas_refine_update(qcd_ctx* c, const float* const* phi, int k, const double* d_gamma, const double* d_rn2,
                       double* x, cudaStream_t s) {
  const long long n = nel<float>(c);
  const unsigned grid = blas_grid(n);
  int done = 0;
  while (done < k) {
    int kk = k - done < 16 ? k - done : 16;
    auto vl = make_list<float>(phi + done, kk);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 16.0 * n * kk + 64.0 * n, 8.0 * c->V * 12 * kk);
    if (kk <= 4)
      refine_update_kernel<4><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, d_rn2, (double2*)x, c->g.Vb, n);
    else if (kk <= 8)
      refine_update_kernel<8><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, d_rn2, (double2*)x, c->g.Vb, n);
    else
      refine_update_kernel<16><<<grid, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, d_rn2, (double2*)x, c->g.Vb,
                                                             n);
    QCD_LAUNCHED();
    done += kk;
  }
  return QCD_OK;
}

int blas_demote_normalised(qcd_ctx* c, const double* r, const double* d_rn2, float* out, cudaStream_t s) {
  const long long n = nel<float>(c);
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 48.0 * n, 0.0);
  demote_normalised_kernel<<<blas_grid(n), kBlasThreads, 0, s>>>((const double2*)r, d_rn2, (float4*)out, c->g.Vb, n);
  QCD_LAUNCHED();
  return QCD_OK;
}

template <typename R>
int blas_norm2(qcd_ctx* c, double* part, const R* v, double* d_out, cudaStream_t s) {
  typedef typename VecT<R>::type E;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, sizeof(E) * (double)n, 4.0 * c->V * 12);
    norm2_kernel<R><<<grid, kBlasThreads, 0, s>>>((const E*)v, n, part);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_out, s);
}

// x /= |x| with |x|^2 taken from the Gram-Schmidt results gs (pass 2 when it
// ran), and the norm stored in *hnorm (the Arnoldi subdiagonal entry)
__global__ void __launch_bounds__(kBlasThreads)
    gs_normalise_kernel(double2* __restrict__ x, const double* __restrict__ gs, int two_pass, double* hnorm,
                        long long n) {
  const double nrm2 = (two_pass && second_pass_needed(gs)) ? gs[4] : gs[1];
  const double nv = sqrt(nrm2);
  if (blockIdx.x == 0 && threadIdx.x == 0) *hnorm = nv;
  const double inv = nv > 0 ? 1.0 / nv : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = rscale(x[i], inv);
}

int blas_gs_normalise(qcd_ctx* c, double* x, const double* d_gs, int two_pass, double* d_hnorm, cudaStream_t s) {
  const long long n = c->V * 12;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 32.0 * n, 2.0 * n);
  gs_normalise_kernel<<<blas_grid(n), kBlasThreads, 0, s>>>((double2*)x, d_gs, two_pass, d_hnorm, n);
  QCD_LAUNCHED();
  return QCD_OK;
}

// CG on the normal equations: alpha = rr / tt;  x += alpha p;  r -= alpha q;
// partial |r|^2
__global__ void __launch_bounds__(kBlasThreads)
    cg_update_kernel(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                     const double2* __restrict__ q, const double* __restrict__ rr, const double* __restrict__ tt,
                     long long n, double* part) {
  const double alpha = *tt > 0 ? *rr / *tt : 0.0;
  double acc[1] = {0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 xi = x[i], ri = r[i];
    const double2 pi = __ldg(p + i), qi = __ldg(q + i);
    xi.x = fma(alpha, pi.x, xi.x);
    xi.y = fma(alpha, pi.y, xi.y);
    ri.x = fma(-alpha, qi.x, ri.x);
    ri.y = fma(-alpha, qi.y, ri.y);
    x[i] = xi;
    r[i] = ri;
    nrm_acc(ri, acc[0]);
  }
  cta_reduce_store<1>(acc, part);
}

// p = r + (rr_new / rr) p
__global__ void __launch_bounds__(kBlasThreads)
    cg_direction_kernel(double2* __restrict__ p, const double2* __restrict__ r, const double* __restrict__ rr_new,
                        const double* __restrict__ rr, long long n) {
  const double beta = *rr > 0 ? *rr_new / *rr : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 ri = __ldg(r + i);
    double2 pi = p[i];
    pi.x = fma(beta, pi.x, ri.x);
    pi.y = fma(beta, pi.y, ri.y);
    p[i] = pi;
  }
}

int blas_cg_update(qcd_ctx* c, double* part, double* x, double* r, const double* p, const double* q,
                   const double* d_rr, const double* d_tt, double* d_rr_new, cudaStream_t s) {
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 96.0 * n, 10.0 * n);
    cg_update_kernel<<<grid, kBlasThreads, 0, s>>>((double2*)x, (double2*)r, (const double2*)p, (const double2*)q,
                                                    d_rr, d_tt, n, part);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_rr_new, s);
}

int blas_cg_direction(qcd_ctx* c, double* p, const double* r, const double* d_rr_new, const double* d_rr,
                      cudaStream_t s) {
  const long long n = c->V * 12;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 48.0 * n, 4.0 * n);
  cg_direction_kernel<<<blas_grid(n), kBlasThreads, 0, s>>>((double2*)p, (const double2*)r, d_rr_new, d_rr, n);
  QCD_LAUNCHED();
  return QCD_OK;
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

#define QCD_BLAS_INST(R)                                                                                              \
  template int blas_multidot<R>(qcd_ctx*, double*, const R* const*, int, const R*, double*, cudaStream_t,            \
                                const double*, double*);                                                              \
  template int blas_axpy_dot<R>(qcd_ctx*, double*, const R* const*, int, const double*, R*, double*, cudaStream_t);  \
  template int blas_axpy_norm_dot<R>(qcd_ctx*, double*, const R* const*, int, const double*, R*, const R*, double*,   \
                                     cudaStream_t, const double*);                                                    \
  template int blas_normalise_update<R>(qcd_ctx*, double*, R*, R*, const double*, int, double*, double*,             \
                                        cudaStream_t);                                                                \
  template int blas_multi_axpy<R>(qcd_ctx*, const R* const*, int, const double*, R*, cudaStream_t);                  \
  template int blas_norm2<R>(qcd_ctx*, double*, const R*, double*, cudaStream_t);
QCD_BLAS_INST(double)
QCD_BLAS_INST(float)
#undef QCD_BLAS_INST

}  // namespace qcd
