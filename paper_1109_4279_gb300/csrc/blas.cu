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

// device side of a Batch: RHS r = blockIdx.y; its vector elements are vs
// elements, its scalars ss doubles and its partial sums ps doubles past RHS 0's
struct BatchDev {
  long long vs, ss, ps;
  const int* mask;
  const int* k;
};

__device__ __forceinline__ bool rhs_skipped(const BatchDev& b) { return b.mask && !b.mask[blockIdx.y]; }

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

__global__ void reduce_partials_kernel(const double* __restrict__ part, int nparts, int stride, int m, double* out,
                                       BatchDev bd) {
  // one warp per value, lanes stride over partials in a fixed order
  if (rhs_skipped(bd)) return;
  part += blockIdx.y * bd.ps;
  out += blockIdx.y * bd.ss;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int l = threadIdx.x & 31;
  if (j >= m) return;
  double t = 0;
  for (int p = l; p < nparts; p += 32) t += part[(long long)p * stride + j];
  t = warp_sum(t);
  if (l == 0) out[j] = t;
}

static BatchDev dev_of(const Batch& B, long long vs) { return BatchDev{vs, B.ss, B.ps, B.mask, B.k}; }

// out[j] = sum_p partials[p * stride + j], j < m (per right-hand side of B)
int reduce_partials(const double* partials, int nparts, int stride, int m, double* out, cudaStream_t s,
                    const Batch& B) {
  const int warps = 8;
  const dim3 grid((m + warps - 1) / warps, B.n);
  reduce_partials_kernel<<<grid, 32 * warps, 0, s>>>(partials, nparts, stride, m, out, dev_of(B, 0));
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
                    const double* cond, double* part, BatchDev bd) {
  typedef typename VecT<R>::type E;
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * bd.vs;
  w += ro;
  if (cond) cond += blockIdx.y * bd.ss;
  part += blockIdx.y * bd.ps;
  if (cond != nullptr && !second_pass_needed(cond)) {  // skipped: zero partial sums, no reduction
    if (threadIdx.x < 2 * K + NORM) part[(long long)blockIdx.x * (2 * K + NORM) + threadIdx.x] = 0.0;
    return;
  }
  R acc[2 * K + NORM];
#pragma unroll
  for (int j = 0; j < 2 * K + NORM; ++j) acc[j] = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const E b = __ldg(w + i);
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) dot_acc(__ldg(vl.v[j] + ro + i), b, acc[2 * j], acc[2 * j + 1]);
    if (NORM) nrm_acc(b, acc[2 * K]);
  }
  cta_reduce_store<2 * K + NORM>(acc, part);
}

// w -= sum_j c_j v_j; then out[j] = (v_j, w) (DOT = 1) or out = {|w|^2, (w, rho)} (DOT = 2)
template <typename R, int K, int DOT>
__global__ void __launch_bounds__(kBlasThreads)
    axpy_dot_kernel(VecList<typename VecT<R>::type> vl, int k, const double* __restrict__ coef,
                    typename VecT<R>::type* __restrict__ w, const typename VecT<R>::type* __restrict__ rho, long long n,
                    const double* cond, double* part, BatchDev bd) {
  typedef typename VecT<R>::type E;
  constexpr int M = DOT == 1 ? 2 * K : 3;
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * bd.vs;
  w += ro;
  if (rho) rho += ro;
  coef += blockIdx.y * bd.ss;
  if (cond) cond += blockIdx.y * bd.ss;
  part += blockIdx.y * bd.ps;
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
        a[j] = __ldg(vl.v[j] + ro + i);
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
                            const double* __restrict__ gs, int two_pass, double* cr, long long n, double* part,
                            BatchDev bd) {
  typedef typename VecT<R>::type E;
  if (rhs_skipped(bd)) return;
  chi += blockIdx.y * bd.vs;
  rho += blockIdx.y * bd.vs;
  gs += blockIdx.y * bd.ss;
  cr += blockIdx.y * bd.ss;
  part += blockIdx.y * bd.ps;
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

// x += sum_j g_j phi_j (j < k, or j < bd.k[r] per right-hand side)
template <typename R, int K>
__global__ void __launch_bounds__(kBlasThreads)
    multi_axpy_kernel(VecList<typename VecT<R>::type> vl, int k, const double* __restrict__ gam,
                      typename VecT<R>::type* __restrict__ x, long long n, BatchDev bd, int koff) {
  typedef typename VecT<R>::type E;
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * bd.vs;
  x += ro;
  gam += blockIdx.y * bd.ss;
  if (bd.k) k = min(k, max(0, bd.k[blockIdx.y] - koff));  // this launch covers vectors koff .. koff + k - 1
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
      if (j < k) cadd(b, cr[j], ci[j], __ldg(vl.v[j] + ro + i));
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
                         double2* __restrict__ x, int Vb, long long n, BatchDev bd, int koff) {
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * bd.vs;
  x += 2 * ro;  // an FP64 field has twice the elements of an FP32 one
  gam += blockIdx.y * bd.ss;
  rn2 += blockIdx.y * bd.ss;
  if (bd.k) k = min(k, max(0, bd.k[blockIdx.y] - koff));  // this launch covers vectors koff .. koff + k - 1
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
      if (j < k) cadd(d, cr[j], ci[j], __ldg(vl.v[j] + ro + i));
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
                             int Vb, long long n, BatchDev bd) {
  if (rhs_skipped(bd)) return;
  r += 2 * blockIdx.y * bd.vs;
  out += blockIdx.y * bd.vs;
  rn2 += blockIdx.y * bd.ss;
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
    norm2_kernel(const typename VecT<R>::type* __restrict__ v, long long n, double* part, BatchDev bd) {
  if (rhs_skipped(bd)) return;
  v += blockIdx.y * bd.vs;
  part += blockIdx.y * bd.ps;
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
__global__ void backsub_kernel(const double* a1, const double* a2, const double* cr, int k, int ld, double* gam,
                               BatchDev bd) {
  // one thread per right-hand side (blockIdx.x)
  if (threadIdx.x != 0) return;
  const int rr = blockIdx.x;
  if (bd.mask && !bd.mask[rr]) return;
  a1 += rr * bd.ss;
  a2 += rr * bd.ss;
  cr += rr * bd.ss;
  gam += rr * bd.ss;
  if (bd.k) k = min(k, bd.k[rr]);
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
// Double-float recursion: vectors of float4 = one complex number as (re hi,
// re lo, im hi, im lo).  A product of two double-floats is split exactly by a
// fused multiply-add, its high part added into a running sum by TwoSum, and
// every lower-order term (the product's error, the cross terms, the sum's
// error) collected in a second FP32 accumulator: 12 FP32 operations per real
// multiply-add instead of one FP64 fused multiply-add, on pipes 64 times
// faster.  Per-thread sums go to FP64 for the CTA and grid reductions.
// ------------------------------------------------------------------------

// (re, im) += conj(a) b
__device__ __forceinline__ void df_dot_acc(const float4& a, const float4& b, dfacc& re, dfacc& im) {
  acc_prod(re, a.x, a.y, b.x, b.y);
  acc_prod(re, a.z, a.w, b.z, b.w);
  acc_prod(im, a.x, a.y, b.z, b.w);
  acc_prod(im, -a.z, -a.w, b.x, b.y);
}
__device__ __forceinline__ void df_nrm_acc(const float4& b, dfacc& n) {
  acc_prod(n, b.x, b.y, b.x, b.y);
  acc_prod(n, b.z, b.w, b.z, b.w);
}
// t = (cr + i ci) a accumulated into (tr, ti)
__device__ __forceinline__ void df_cmul_acc(df cr, df ci, const float4& a, dfacc& tr, dfacc& ti) {
  acc_prod(tr, cr.hi, cr.lo, a.x, a.y);
  acc_prod(tr, -ci.hi, -ci.lo, a.z, a.w);
  acc_prod(ti, cr.hi, cr.lo, a.z, a.w);
  acc_prod(ti, ci.hi, ci.lo, a.x, a.y);
}
// b - (tr, ti) as a double-float complex element
__device__ __forceinline__ float4 df_csub(const float4& b, const dfacc& tr, const dfacc& ti) {
  const df re = df_add(df{b.x, b.y}, df_neg(acc_df(tr)));
  const df im = df_add(df{b.z, b.w}, df_neg(acc_df(ti)));
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

template <int M>
__device__ __forceinline__ void df_reduce_store(const dfacc (&a)[M], double* part) {
  double v[M];
#pragma unroll
  for (int j = 0; j < M; ++j) v[j] = acc_value(a[j]);
  cta_reduce_store<M>(v, part);
}

// out[j] = (v_j, w), j < k <= K; with NORM also |w|^2 (as multidot_kernel)
template <int K, int NORM>
__global__ void __launch_bounds__(kBlasThreads)
    df_multidot_kernel(VecList<float4> vl, int k, const float4* __restrict__ w, long long n, const double* cond,
                       double* part, BatchDev bd) {
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * bd.vs;
  w += ro;
  if (cond) cond += blockIdx.y * bd.ss;
  part += blockIdx.y * bd.ps;
  if (cond != nullptr && !second_pass_needed(cond)) {  // skipped: zero partial sums, no reduction
    if (threadIdx.x < 2 * K + NORM) part[(long long)blockIdx.x * (2 * K + NORM) + threadIdx.x] = 0.0;
    return;
  }
  dfacc acc[2 * K + NORM];
#pragma unroll
  for (int j = 0; j < 2 * K + NORM; ++j) acc[j] = {0.f, 0.f};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 b = __ldg(w + i);
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) df_dot_acc(__ldg(vl.v[j] + ro + i), b, acc[2 * j], acc[2 * j + 1]);
    if (NORM) df_nrm_acc(b, acc[2 * K]);
  }
  df_reduce_store<2 * K + NORM>(acc, part);
}

// w -= sum_j c_j v_j; then {|w|^2, (w, rho)} (as axpy_dot_kernel with DOT = 2)
template <int K>
__global__ void __launch_bounds__(kBlasThreads)
    df_axpy_norm_dot_kernel(VecList<float4> vl, int k, const double* __restrict__ coef, float4* __restrict__ w,
                            const float4* __restrict__ rho, long long n, const double* cond, double* part,
                            BatchDev bd) {
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * bd.vs;
  w += ro;
  rho += ro;
  coef += blockIdx.y * bd.ss;
  if (cond) cond += blockIdx.y * bd.ss;
  part += blockIdx.y * bd.ps;
  if (cond != nullptr && !second_pass_needed(cond)) return;  // block-uniform: no partials written
  df cr[K], ci[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    cr[j] = j < k ? df_from_f64(coef[2 * j]) : df{0.f, 0.f};
    ci[j] = j < k ? df_from_f64(coef[2 * j + 1]) : df{0.f, 0.f};
  }
  dfacc acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float4 b = w[i];
    if (k > 0) {
      dfacc tr = {0.f, 0.f}, ti = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < k) df_cmul_acc(cr[j], ci[j], __ldg(vl.v[j] + ro + i), tr, ti);
      b = df_csub(b, tr, ti);
      w[i] = b;
    }
    df_nrm_acc(b, acc[0]);
    df_dot_acc(b, __ldg(rho + i), acc[1], acc[2]);
  }
  df_reduce_store<3>(acc, part);
}

// as normalise_update_kernel: chi /= |chi|; rho -= ((chi, rho) / |chi|^2) chi_unnormalised; |rho|^2
__global__ void __launch_bounds__(kBlasThreads)
    df_normalise_update_kernel(float4* __restrict__ chi, float4* __restrict__ rho, const double* __restrict__ gs,
                               int two_pass, double* cr, long long n, double* part, BatchDev bd) {
  if (rhs_skipped(bd)) return;
  chi += blockIdx.y * bd.vs;
  rho += blockIdx.y * bd.vs;
  gs += blockIdx.y * bd.ss;
  cr += blockIdx.y * bd.ss;
  part += blockIdx.y * bd.ps;
  const double* co = (two_pass && second_pass_needed(gs)) ? gs + 4 : gs + 1;
  const double nrm2 = co[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cr[0] = co[0];
    cr[1] = co[1];
    cr[2] = co[2];
  }
  const df inv = df_from_f64(nrm2 > 0 ? 1.0 / sqrt(nrm2) : 0.0);
  const df cre = df_from_f64(nrm2 > 0 ? co[1] / nrm2 : 0.0), cim = df_from_f64(nrm2 > 0 ? co[2] / nrm2 : 0.0);
  dfacc acc[1] = {{0.f, 0.f}};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 x = chi[i];
    dfacc tr = {0.f, 0.f}, ti = {0.f, 0.f};
    df_cmul_acc(cre, cim, x, tr, ti);
    const float4 r = df_csub(rho[i], tr, ti);
    rho[i] = r;
    const df xr = df_mul(df{x.x, x.y}, inv), xi = df_mul(df{x.z, x.w}, inv);
    chi[i] = make_float4(xr.hi, xr.lo, xi.hi, xi.lo);
    df_nrm_acc(r, acc[0]);
  }
  df_reduce_store<1>(acc, part);
}

// x64 += sum_j g_j phi_j with double-float phi_j: the sum formed in
// double-float arithmetic, added to the FP64 solution once (one FP64 addition
// per real instead of 4 k fused multiply-adds)
template <int K>
__global__ void __launch_bounds__(kBlasThreads)
    df_update_kernel(VecList<float4> vl, int k, const double* __restrict__ gam, double2* __restrict__ x, long long n,
                     BatchDev bd, int koff) {
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * bd.vs;
  x += ro;
  gam += blockIdx.y * bd.ss;
  if (bd.k) k = min(k, max(0, bd.k[blockIdx.y] - koff));
  df gr[K], gi[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    gr[j] = j < k ? df_from_f64(gam[2 * j]) : df{0.f, 0.f};
    gi[j] = j < k ? df_from_f64(gam[2 * j + 1]) : df{0.f, 0.f};
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    dfacc tr = {0.f, 0.f}, ti = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) df_cmul_acc(gr[j], gi[j], __ldg(vl.v[j] + ro + i), tr, ti);
    double2 v = x[i];
    v.x += acc_value(tr);
    v.y += acc_value(ti);
    x[i] = v;
  }
}

// the same update from FP32 phi_j (FP32-exact preconditioner outputs): each
// float4 of a phi field holds complexes 2 c, 2 c + 1 of site (blk, r) -- chunk
// (blk * 6 + c) Vb + r -- which are elements (blk * 12 + 2 c) Vb + r and the next
// chunk row of x; the products are those of the double-float form with zero
// low parts
template <int K>
__global__ void __launch_bounds__(kBlasThreads)
    df_update32_kernel(VecList<float4> vl, int k, const double* __restrict__ gam, double2* __restrict__ x,
                       long long nchunk, int Vb, BatchDev bd, int koff, float4* __restrict__ xs) {
  if (rhs_skipped(bd)) return;
  const long long ro = blockIdx.y * (bd.vs / 2);  // phi: half the float4 elements of an x-sized field
  x += blockIdx.y * bd.vs;
  if (xs) xs += blockIdx.y * bd.vs;
  gam += blockIdx.y * bd.ss;
  if (bd.k) k = min(k, max(0, bd.k[blockIdx.y] - koff));
  df gr[K], gi[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    gr[j] = j < k ? df_from_f64(gam[2 * j]) : df{0.f, 0.f};
    gi[j] = j < k ? df_from_f64(gam[2 * j + 1]) : df{0.f, 0.f};
  }
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < nchunk;
       m += (long long)gridDim.x * blockDim.x) {
    const long long t = m / Vb;
    const int r = (int)(m - t * Vb), cc = (int)(t % 6);
    const long long blk = t / 6;
    const long long i0 = (blk * 12 + 2 * cc) * Vb + r;
    dfacc tr0 = {0.f, 0.f}, ti0 = {0.f, 0.f}, tr1 = {0.f, 0.f}, ti1 = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) {
        const float4 p = __ldg(vl.v[j] + ro + m);
        df_cmul_acc(gr[j], gi[j], make_float4(p.x, 0.f, p.y, 0.f), tr0, ti0);
        df_cmul_acc(gr[j], gi[j], make_float4(p.z, 0.f, p.w, 0.f), tr1, ti1);
      }
    double2 v = x[i0];
    v.x += acc_value(tr0);
    v.y += acc_value(ti0);
    x[i0] = v;
    if (xs) {  // the updated x's double-float split too (same element order)
      const df a = df_from_f64(v.x), b = df_from_f64(v.y);
      xs[i0] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    v = x[i0 + Vb];
    v.x += acc_value(tr1);
    v.y += acc_value(ti1);
    x[i0 + Vb] = v;
    if (xs) {
      const df a = df_from_f64(v.x), b = df_from_f64(v.y);
      xs[i0 + Vb] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
  }
}

// out = the double-float split of an FP64 field (same element order)
__global__ void __launch_bounds__(kBlasThreads)
    df_split_kernel(const double2* __restrict__ in, float4* __restrict__ out, long long n, BatchDev bd) {
  if (rhs_skipped(bd)) return;
  in += blockIdx.y * bd.vs;
  out += blockIdx.y * bd.vs;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = __ldg(in + i);
    const df a = df_from_f64(v.x), b = df_from_f64(v.y);
    out[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
  }
}

// out = the FP64 value of a double-float field (same element order)
__global__ void __launch_bounds__(kBlasThreads)
    df_join_kernel(const float4* __restrict__ in, double2* __restrict__ out, long long n, BatchDev bd) {
  if (rhs_skipped(bd)) return;
  in += blockIdx.y * bd.vs;
  out += blockIdx.y * bd.vs;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = __ldg(in + i);
    out[i] = make_double2(df_to_f64(df{v.x, v.y}), df_to_f64(df{v.z, v.w}));
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
                  const double* cond, double* d_norm, const Batch& B) {
  typedef typename VecT<R>::type E;
  if (k <= 0) return QCD_OK;
  if (k > kMaxVec) return QCD_ERR_ARG;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  // a conditional (second Gram-Schmidt) pass is counted as no work: the host
  // cannot know whether it runs, and on well-conditioned bases it returns at once
  const double work = (cond ? 0.0 : 1.0) * B.n;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, work * sizeof(E) * (double)n * (k + 1), work * 8.0 * c->V * 12 * k);
  const int K = pick_k(k);
  const BatchDev bd = dev_of(B, n);
  int done = 0;
  while (done < k) {
    const int kk = k - done < K ? k - done : K;
    const int norm = (d_norm != nullptr && done == 0) ? 1 : 0;
    const int M = 2 * K + norm;
    auto vl = make_list<R>(v + done, kk);
    const E* w2 = (const E*)w;
    const dim3 g2(grid, B.n);
#define MD(KK)                                                                           \
  if (norm)                                                                              \
    multidot_kernel<R, KK, 1><<<g2, kBlasThreads, 0, s>>>(vl, kk, w2, n, cond, part, bd); \
  else                                                                                   \
    multidot_kernel<R, KK, 0><<<g2, kBlasThreads, 0, s>>>(vl, kk, w2, n, cond, part, bd);
    switch (K) {
      case 4: MD(4); break;
      case 8: MD(8); break;
      case 16: MD(16); break;
      default: MD(32); break;
    }
#undef MD
    QCD_LAUNCHED();
    QCD_TRY(reduce_partials(part, (int)grid, M, 2 * kk, d_out + 2 * done, s, B));
    if (norm) QCD_TRY(reduce_partials(part + 2 * K, (int)grid, M, 1, d_norm, s, B));
    done += kk;
  }
  return QCD_OK;
}

template <typename R, int DOT>
static int axpy_dot_impl(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, const R* rho,
                         double* d_out, cudaStream_t s, const double* cond, const Batch& B) {
  typedef typename VecT<R>::type E;
  if (k > 32) return QCD_ERR_UNSUPPORTED;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  const int K = pick_k(k);
  const int M = DOT == 1 ? 2 * K : 3;
  const double work = (cond ? 0.0 : 1.0) * B.n;  // conditional pass: counted as no work (see blas_multidot)
  ProfScope ps(c, QCD_KERNEL_BLAS, s, work * sizeof(E) * (double)n * (k + 2 + (DOT == 2)),
               work * 16.0 * c->V * 12 * k);
  auto vl = make_list<R>(v, k);
  const E* r2 = (const E*)rho;
  E* w2 = (E*)w;
  const dim3 g2(grid, B.n);
  const BatchDev bd = dev_of(B, n);
  switch (K) {
    case 4: axpy_dot_kernel<R, 4, DOT><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part, bd); break;
    case 8: axpy_dot_kernel<R, 8, DOT><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part, bd); break;
    case 16: axpy_dot_kernel<R, 16, DOT><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part, bd); break;
    default: axpy_dot_kernel<R, 32, DOT><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w2, r2, n, cond, part, bd); break;
  }
  QCD_LAUNCHED();
  return reduce_partials(part, (int)grid, M, DOT == 1 ? 2 * k : 3, d_out, s, B);
}

template <typename R>
int blas_axpy_dot(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, double* d_out,
                  cudaStream_t s, const Batch& B) {
  if (k <= 0) return QCD_OK;
  return axpy_dot_impl<R, 1>(c, part, v, k, d_coef, w, nullptr, d_out, s, nullptr, B);
}

template <typename R>
int blas_axpy_norm_dot(qcd_ctx* c, double* part, const R* const* v, int k, const double* d_coef, R* w, const R* rho,
                       double* d_out, cudaStream_t s, const double* cond, const Batch& B) {
  typedef typename VecT<R>::type E;
  if (k <= 0) {
    // nothing to subtract: only the norm and the dot
    const long long n = nel<R>(c);
    const unsigned grid = blas_grid(n);
    auto vl = make_list<R>(v, 0);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 2.0 * sizeof(E) * n * B.n, 8.0 * c->V * 12 * B.n);
    axpy_dot_kernel<R, 4, 2><<<dim3(grid, B.n), kBlasThreads, 0, s>>>(vl, 0, d_coef, (E*)w, (const E*)rho, n, cond,
                                                                       part, dev_of(B, n));
    QCD_LAUNCHED();
    return reduce_partials(part, (int)grid, 3, 3, d_out, s, B);
  }
  return axpy_dot_impl<R, 2>(c, part, v, k, d_coef, w, rho, d_out, s, cond, B);
}

template <typename R>
int blas_normalise_update(qcd_ctx* c, double* part, R* chi, R* rho, const double* d_gs, int two_pass, double* d_cr,
                          double* d_out, cudaStream_t s, const Batch& B) {
  typedef typename VecT<R>::type E;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 4.0 * sizeof(E) * n * B.n, 8.0 * c->V * 12 * B.n);
    normalise_update_kernel<R><<<dim3(grid, B.n), kBlasThreads, 0, s>>>((E*)chi, (E*)rho, d_gs, two_pass, d_cr, n,
                                                                         part, dev_of(B, n));
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_out, s, B);
}

template <typename R>
int blas_multi_axpy(qcd_ctx* c, const R* const* phi, int k, const double* d_gamma, R* x, cudaStream_t s,
                    const Batch& B) {
  typedef typename VecT<R>::type E;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  const dim3 g2(grid, B.n);
  int done = 0;
  while (done < k) {
    int kk = k - done < 16 ? k - done : 16;
    auto vl = make_list<R>(phi + done, kk);
    const BatchDev bd = dev_of(B, n);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, sizeof(E) * (double)n * (kk + 2) * B.n, 8.0 * c->V * 12 * kk * B.n);
    if (kk <= 4)
      multi_axpy_kernel<R, 4><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (E*)x, n, bd, done);
    else if (kk <= 8)
      multi_axpy_kernel<R, 8><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (E*)x, n, bd, done);
    else
      multi_axpy_kernel<R, 16><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (E*)x, n, bd, done);
    QCD_LAUNCHED();
    done += kk;
  }
  return QCD_OK;
}

int blas_refine_update(qcd_ctx* c, const float* const* phi, int k, const double* d_gamma, const double* d_rn2,
                       double* x, cudaStream_t s, const Batch& B) {
  const long long n = nel<float>(c);
  const unsigned grid = blas_grid(n);
  const dim3 g2(grid, B.n);
  const BatchDev bd = dev_of(B, n);
  int done = 0;
  while (done < k) {
    int kk = k - done < 16 ? k - done : 16;
    auto vl = make_list<float>(phi + done, kk);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, (16.0 * n * kk + 64.0 * n) * B.n, 8.0 * c->V * 12 * kk * B.n);
    if (kk <= 4)
      refine_update_kernel<4><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, d_rn2, (double2*)x, c->g.Vb, n,
                                                          bd, done);
    else if (kk <= 8)
      refine_update_kernel<8><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, d_rn2, (double2*)x, c->g.Vb, n,
                                                          bd, done);
    else
      refine_update_kernel<16><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, d_rn2, (double2*)x, c->g.Vb,
                                                           n, bd, done);
    QCD_LAUNCHED();
    done += kk;
  }
  return QCD_OK;
}

int blas_demote_normalised(qcd_ctx* c, const double* r, const double* d_rn2, float* out, cudaStream_t s,
                           const Batch& B) {
  const long long n = nel<float>(c);
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 48.0 * n * B.n, 0.0);
  demote_normalised_kernel<<<dim3(blas_grid(n), B.n), kBlasThreads, 0, s>>>((const double2*)r, d_rn2, (float4*)out,
                                                                              c->g.Vb, n, dev_of(B, n));
  QCD_LAUNCHED();
  return QCD_OK;
}

template <typename R>
int blas_norm2(qcd_ctx* c, double* part, const R* v, double* d_out, cudaStream_t s, const Batch& B) {
  typedef typename VecT<R>::type E;
  const long long n = nel<R>(c);
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, sizeof(E) * (double)n * B.n, 4.0 * c->V * 12 * B.n);
    norm2_kernel<R><<<dim3(grid, B.n), kBlasThreads, 0, s>>>((const E*)v, n, part, dev_of(B, n));
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_out, s, B);
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
                 cudaStream_t s, const Batch& B) {
  backsub_kernel<<<B.n, 32, 0, s>>>(d_a1, d_a2, d_cr, k, ld, d_gamma, dev_of(B, 0));
  QCD_LAUNCHED();
  return QCD_OK;
}

// ---- double-float recursion (fields of V * 12 float4 per right-hand side)
static VecList<float4> make_df_list(const float4* const* v, int k) {
  VecList<float4> vl;
  for (int j = 0; j < kMaxVec; ++j) vl.v[j] = j < k ? v[j] : nullptr;
  return vl;
}

int blas_df_multidot(qcd_ctx* c, double* part, const float4* const* v, int k, const float4* w, double* d_out,
                     cudaStream_t s, const double* cond, double* d_norm, const Batch& B) {
  if (k <= 0) return QCD_OK;
  if (k > kMaxVec) return QCD_ERR_ARG;
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  const double work = (cond ? 0.0 : 1.0) * B.n;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, work * 16.0 * (double)n * (k + 1), work * 8.0 * c->V * 12 * k);
  const int K = pick_k(k) > 16 ? 16 : pick_k(k);
  const BatchDev bd = dev_of(B, n);
  const dim3 g2(grid, B.n);
  int done = 0;
  while (done < k) {
    const int kk = k - done < K ? k - done : K;
    const int norm = (d_norm != nullptr && done == 0) ? 1 : 0;
    const int M = 2 * K + norm;
    auto vl = make_df_list(v + done, kk);
#define MD(KK)                                                                        \
  if (norm)                                                                           \
    df_multidot_kernel<KK, 1><<<g2, kBlasThreads, 0, s>>>(vl, kk, w, n, cond, part, bd); \
  else                                                                                \
    df_multidot_kernel<KK, 0><<<g2, kBlasThreads, 0, s>>>(vl, kk, w, n, cond, part, bd);
    switch (K) {
      case 4: MD(4); break;
      case 8: MD(8); break;
      default: MD(16); break;
    }
#undef MD
    QCD_LAUNCHED();
    QCD_TRY(reduce_partials(part, (int)grid, M, 2 * kk, d_out + 2 * done, s, B));
    if (norm) QCD_TRY(reduce_partials(part + 2 * K, (int)grid, M, 1, d_norm, s, B));
    done += kk;
  }
  return QCD_OK;
}

int blas_df_axpy_norm_dot(qcd_ctx* c, double* part, const float4* const* v, int k, const double* d_coef, float4* w,
                          const float4* rho, double* d_out, cudaStream_t s, const double* cond, const Batch& B) {
  if (k > 32) return QCD_ERR_UNSUPPORTED;
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  const int K = k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 16 ? 16 : 32));
  const double work = (cond ? 0.0 : 1.0) * B.n;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, work * 16.0 * (double)n * (k + 3), work * 16.0 * c->V * 12 * (k + 1));
  auto vl = make_df_list(v, k);
  const dim3 g2(grid, B.n);
  const BatchDev bd = dev_of(B, n);
  switch (K) {
    case 4: df_axpy_norm_dot_kernel<4><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w, rho, n, cond, part, bd); break;
    case 8: df_axpy_norm_dot_kernel<8><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w, rho, n, cond, part, bd); break;
    case 16: df_axpy_norm_dot_kernel<16><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w, rho, n, cond, part, bd); break;
    default: df_axpy_norm_dot_kernel<32><<<g2, kBlasThreads, 0, s>>>(vl, k, d_coef, w, rho, n, cond, part, bd); break;
  }
  QCD_LAUNCHED();
  return reduce_partials(part, (int)grid, 3, 3, d_out, s, B);
}

int blas_df_normalise_update(qcd_ctx* c, double* part, float4* chi, float4* rho, const double* d_gs, int two_pass,
                             double* d_cr, double* d_out, cudaStream_t s, const Batch& B) {
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  {
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 64.0 * n * B.n, 8.0 * c->V * 12 * B.n);
    df_normalise_update_kernel<<<dim3(grid, B.n), kBlasThreads, 0, s>>>(chi, rho, d_gs, two_pass, d_cr, n, part,
                                                                         dev_of(B, n));
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_out, s, B);
}

int blas_df_update(qcd_ctx* c, const float4* const* phi, int k, const double* d_gamma, double* x, cudaStream_t s,
                   const Batch& B) {
  const long long n = c->V * 12;
  const unsigned grid = blas_grid(n);
  const dim3 g2(grid, B.n);
  const BatchDev bd = dev_of(B, n);
  int done = 0;
  while (done < k) {
    const int kk = k - done < 16 ? k - done : 16;
    auto vl = make_df_list(phi + done, kk);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, 16.0 * (double)n * (kk + 2) * B.n, 8.0 * c->V * 12 * kk * B.n);
    if (kk <= 4)
      df_update_kernel<4><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, n, bd, done);
    else if (kk <= 8)
      df_update_kernel<8><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, n, bd, done);
    else
      df_update_kernel<16><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, n, bd, done);
    QCD_LAUNCHED();
    done += kk;
  }
  return QCD_OK;
}

int blas_df_update32(qcd_ctx* c, const float4* const* phi, int k, const double* d_gamma, double* x, cudaStream_t s,
                     const Batch& B, float* xs) {
  const long long n = c->V * 12, nchunk = c->V * 6;
  const dim3 g2(blas_grid(nchunk), B.n);
  const BatchDev bd = dev_of(B, n);
  const int Vb = c->g.Vb;
  int done = 0;
  while (done < k) {
    const int kk = k - done < 16 ? k - done : 16;
    auto vl = make_df_list(phi + done, kk);
    ProfScope ps(c, QCD_KERNEL_BLAS, s, (8.0 * kk + 32.0) * (double)n * B.n, 8.0 * c->V * 12 * kk * B.n);
    float4* x4 = done + kk == k ? (float4*)xs : nullptr;  // the split after the last part of the update
    if (kk <= 4)
      df_update32_kernel<4><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, nchunk, Vb, bd, done,
                                                         x4);
    else if (kk <= 8)
      df_update32_kernel<8><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, nchunk, Vb, bd, done,
                                                         x4);
    else
      df_update32_kernel<16><<<g2, kBlasThreads, 0, s>>>(vl, kk, d_gamma + 2 * done, (double2*)x, nchunk, Vb, bd,
                                                          done, x4);
    QCD_LAUNCHED();
    done += kk;
  }
  return QCD_OK;
}

int blas_df_split(qcd_ctx* c, const double* in, float* out, cudaStream_t s, const Batch& B) {
  const long long n = c->V * 12;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 32.0 * n * B.n, 0.0);
  df_split_kernel<<<dim3(blas_grid(n), B.n), kBlasThreads, 0, s>>>((const double2*)in, (float4*)out, n,
                                                                    dev_of(B, n));
  QCD_LAUNCHED();
  return QCD_OK;
}

int blas_df_join(qcd_ctx* c, const float* in, double* out, cudaStream_t s, const Batch& B) {
  const long long n = c->V * 12;
  ProfScope ps(c, QCD_KERNEL_BLAS, s, 32.0 * n * B.n, 0.0);
  df_join_kernel<<<dim3(blas_grid(n), B.n), kBlasThreads, 0, s>>>((const float4*)in, (double2*)out, n,
                                                                   dev_of(B, n));
  QCD_LAUNCHED();
  return QCD_OK;
}

#define QCD_BLAS_INST(R)                                                                                              \
  template int blas_multidot<R>(qcd_ctx*, double*, const R* const*, int, const R*, double*, cudaStream_t,            \
                                const double*, double*, const Batch&);                                                \
  template int blas_axpy_dot<R>(qcd_ctx*, double*, const R* const*, int, const double*, R*, double*, cudaStream_t,   \
                                const Batch&);                                                                        \
  template int blas_axpy_norm_dot<R>(qcd_ctx*, double*, const R* const*, int, const double*, R*, const R*, double*,   \
                                     cudaStream_t, const double*, const Batch&);                                      \
  template int blas_normalise_update<R>(qcd_ctx*, double*, R*, R*, const double*, int, double*, double*,             \
                                        cudaStream_t, const Batch&);                                                  \
  template int blas_multi_axpy<R>(qcd_ctx*, const R* const*, int, const double*, R*, cudaStream_t, const Batch&);    \
  template int blas_norm2<R>(qcd_ctx*, double*, const R*, double*, cudaStream_t, const Batch&);
QCD_BLAS_INST(double)
QCD_BLAS_INST(float)
#undef QCD_BLAS_INST

}  // namespace qcd
