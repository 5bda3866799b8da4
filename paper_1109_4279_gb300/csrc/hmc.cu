// Hybrid Monte Carlo molecular dynamics for two degenerate clover-Wilson
// flavours (Sec. 1: the inversions exist to feed the HMC fermion force).
//
// Gauge fields are lexicographic FP64 device arrays (V,4,3,3) complex, the
// layout qcd_load_gauge takes; momenta and forces are (V,4,8) FP64 with
// P = sum_a pi_a lambda_a / 2, derivatives taken for
// U_mu(x) -> exp(i theta_a lambda_a / 2) U_mu(x).
//   S_g = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3)          (plaquettes)
//   dS_g/dtheta_a = (beta / 6) Im tr(lambda_a U_mu(x) V_mu(x))     (V: six staples)
//   S_f = phi^+ (D^+ D)^-1 phi = |Y|^2, Y = D^-+ phi, phi = D^+ eta
//   dS_f/dtheta_a = -2 Re(Y^+ dD/dtheta_a X), X = D^-1 Y            (qcd_force)
// Leapfrog: pi -= eps/2 F; n times {U <- exp(i eps P) U; pi -= eps F} with a
// final half step; Metropolis accepts when u < exp(-dH).
#include <cmath>
#include <cstring>

#include "internal.h"

namespace qcd {

typedef cpx<double> cd;

struct M3 {
  cd a[3][3];
};

__device__ __forceinline__ M3 mload(const double2* U, long long link) {
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 v = U[link * 9 + k];
    m.a[k / 3][k % 3] = {v.x, v.y};
  }
  return m;
}
__device__ __forceinline__ void mstore(double2* U, long long link, const M3& m) {
#pragma unroll
  for (int k = 0; k < 9; ++k) U[link * 9 + k] = make_double2(m.a[k / 3][k % 3].re, m.a[k / 3][k % 3].im);
}
__device__ __forceinline__ M3 mmul(const M3& x, const M3& y) {
  M3 z;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd s = cmul(x.a[i][0], y.a[0][j]);
      s = cmadd(x.a[i][1], y.a[1][j], s);
      s = cmadd(x.a[i][2], y.a[2][j], s);
      z.a[i][j] = s;
    }
  return z;
}
__device__ __forceinline__ M3 mdag(const M3& x) {
  M3 z;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) z.a[i][j] = conjg(x.a[j][i]);
  return z;
}
__device__ __forceinline__ void madd(M3& x, const M3& y) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) x.a[i][j] = x.a[i][j] + y.a[i][j];
}

struct Lex {
  int L[4];
  long long V;
  __device__ __forceinline__ void coords(long long s, int x[4]) const {
#pragma unroll
    for (int mu = 3; mu >= 0; --mu) {
      x[mu] = (int)(s % L[mu]);
      s /= L[mu];
    }
  }
  __device__ __forceinline__ long long index(const int x[4]) const {
    return (((long long)x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3];
  }
  // site s shifted by d (+-1) in direction mu, periodic (the gauge field is periodic)
  __device__ __forceinline__ long long shift(long long s, int mu, int d) const {
    int x[4];
    coords(s, x);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu)
      if (nu == mu) x[nu] = (x[nu] + d + L[nu]) % L[nu];
    return index(x);
  }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// per-CTA sum in a fixed order (256 threads); part[blockIdx.x]
__device__ __forceinline__ void cta_sum_store(double v, double* part) {
  __shared__ double sh[8];
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    part[blockIdx.x] = t;
  }
}

static const int kThreads = 256;

// V_mu(x) = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
__device__ M3 staple_sum(const Lex& g, const double2* U, long long s, int mu) {
  M3 v;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) v.a[i][j] = {0, 0};
  const long long sp = g.shift(s, mu, +1);
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const long long sn = g.shift(s, nu, +1), sm = g.shift(s, nu, -1);
    const long long spm = g.shift(sp, nu, -1);
    madd(v, mmul(mmul(mload(U, sp * 4 + nu), mdag(mload(U, sn * 4 + mu))), mdag(mload(U, s * 4 + nu))));
    madd(v, mmul(mmul(mdag(mload(U, spm * 4 + nu)), mdag(mload(U, sm * 4 + mu))), mload(U, sm * 4 + nu)));
  }
  return v;
}

// F_a = (beta / 6) Im tr(lambda_a M), M = U_mu(x) V_mu(x); tr(lambda_a M) written out
__global__ void __launch_bounds__(kThreads) gauge_force_kernel(Lex g, const double2* __restrict__ U, double beta,
                                                               double* __restrict__ F) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * g.V) return;
  const long long s = l / 4;
  const int mu = (int)(l % 4);
  const M3 M = mmul(mload(U, l), staple_sum(g, U, s, mu));
  const double f = beta / 6.0, r3 = 0.5773502691896257645;  // 1/sqrt(3)
  double* o = F + l * 8;
  o[0] = f * (M.a[1][0].im + M.a[0][1].im);                         // tr(l1 M) = M10 + M01
  o[1] = f * (M.a[0][1].re - M.a[1][0].re);                         // tr(l2 M) = i (M01 - M10)
  o[2] = f * (M.a[0][0].im - M.a[1][1].im);                         // tr(l3 M) = M00 - M11
  o[3] = f * (M.a[2][0].im + M.a[0][2].im);                         // tr(l4 M) = M20 + M02
  o[4] = f * (M.a[0][2].re - M.a[2][0].re);                         // tr(l5 M) = i (M02 - M20)
  o[5] = f * (M.a[2][1].im + M.a[1][2].im);                         // tr(l6 M) = M21 + M12
  o[6] = f * (M.a[1][2].re - M.a[2][1].re);                         // tr(l7 M) = i (M12 - M21)
  o[7] = f * r3 * (M.a[0][0].im + M.a[1][1].im - 2.0 * M.a[2][2].im);  // tr(l8 M)
}

// per site: sum over mu < nu of (1 - Re tr U_munu / 3); partial sums per CTA
__global__ void __launch_bounds__(kThreads) plaquette_kernel(Lex g, const double2* __restrict__ U, double* part) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0;
  if (s < g.V) {
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      const long long smu = g.shift(s, mu, +1);
      const M3 Um = mload(U, s * 4 + mu);
#pragma unroll 1
      for (int nu = mu + 1; nu < 4; ++nu) {
        const long long snu = g.shift(s, nu, +1);
        const M3 P = mmul(mmul(Um, mload(U, smu * 4 + nu)), mdag(mmul(mload(U, s * 4 + nu), mload(U, snu * 4 + mu))));
        acc += 1.0 - (P.a[0][0].re + P.a[1][1].re + P.a[2][2].re) / 3.0;
      }
    }
  }
  cta_sum_store(acc, part);
}

// exp(A) of a small 3x3 complex matrix: Taylor series of A / 2^k to order 14
// (|A / 2^k| <= 1/4 in the Frobenius norm, truncation below 1e-18), then k squarings
__device__ M3 mexp(M3 A) {
  double n2 = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) n2 += A.a[i][j].re * A.a[i][j].re + A.a[i][j].im * A.a[i][j].im;
  double nrm = sqrt(n2);
  int k = 0;
  while (nrm > 0.25 && k < 60) {
    nrm *= 0.5;
    ++k;
  }
  const double sc = ldexp(1.0, -k);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A.a[i][j] = sc * A.a[i][j];
  // Horner: E = I + A (I + A/2 (I + A/3 (... (I + A/14))))
  M3 E;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) E.a[i][j] = {i == j ? 1.0 : 0.0, 0.0};
  for (int t = 14; t >= 1; --t) {
    M3 T = mmul(A, E);
    const double inv = 1.0 / t;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) E.a[i][j] = {(i == j ? 1.0 : 0.0) + inv * T.a[i][j].re, inv * T.a[i][j].im};
  }
  for (int q = 0; q < k; ++q) E = mmul(E, E);
  return E;
}

// U_mu(x) <- exp(i eps P) U_mu(x), P = sum_a pi_a lambda_a / 2
__global__ void __launch_bounds__(kThreads) link_update_kernel(long long nlinks, double2* __restrict__ U,
                                                               const double* __restrict__ pi, double eps) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlinks) return;
  const double* p = pi + l * 8;
  const double h = 0.5 * eps, r3 = 0.5773502691896257645;
  // i eps P with P Hermitian: P00 = (p3 + p8/sqrt3)/2, P11 = (-p3 + p8/sqrt3)/2, P22 = -p8/sqrt3,
  // P01 = (p1 - i p2)/2, P02 = (p4 - i p5)/2, P12 = (p6 - i p7)/2, P10 = conj(P01), ...
  M3 A;
  const double d0 = h * (p[2] + r3 * p[7]), d1 = h * (-p[2] + r3 * p[7]), d2 = -h * 2.0 * r3 * p[7];
  A.a[0][0] = {0, d0};
  A.a[1][1] = {0, d1};
  A.a[2][2] = {0, d2};
  // i (x - i y) = y + i x;  i (x + i y) = -y + i x
  A.a[0][1] = {h * p[1], h * p[0]};
  A.a[1][0] = {-h * p[1], h * p[0]};
  A.a[0][2] = {h * p[4], h * p[3]};
  A.a[2][0] = {-h * p[4], h * p[3]};
  A.a[1][2] = {h * p[6], h * p[5]};
  A.a[2][1] = {-h * p[6], h * p[5]};
  mstore(U, l, mmul(mexp(A), mload(U, l)));
}

// pi -= step (Fg + cf Ff)
__global__ void __launch_bounds__(kThreads) momentum_update_kernel(long long n, double* __restrict__ pi,
                                                                   const double* __restrict__ Fg,
                                                                   const double* __restrict__ Ff, double cf,
                                                                   double step) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pi[i] -= step * (Fg[i] + cf * Ff[i]);
}

__global__ void __launch_bounds__(kThreads) sumsq_kernel(long long n, const double* __restrict__ v, double* part) {
  double acc = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc = fma(v[i], v[i], acc);
  cta_sum_store(acc, part);
}

static Lex lex_of(qcd_ctx* c) {
  Lex g;
  for (int mu = 0; mu < 4; ++mu) g.L[mu] = c->p.dims[mu];
  g.V = c->V;
  return g;
}

static unsigned grid_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// device scratch for partial sums (one per CTA of the widest kernel) and one result
struct HmcScratch {
  double* part = nullptr;
  double* res = nullptr;
  size_t nparts = 0;
  ~HmcScratch() {
    if (part) cudaFree(part);
    if (res) cudaFree(res);
  }
  int init(long long V) {
    nparts = grid_for(V * 4);
    if (cudaMalloc(&part, sizeof(double) * nparts) != cudaSuccess || cudaMalloc(&res, sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return QCD_ERR_NOMEM;
    }
    return QCD_OK;
  }
};

static int sum_to_host(const double* part, int nparts, double* d_res, double* out, cudaStream_t s) {
  QCD_TRY(reduce_partials(part, nparts, 1, 1, d_res, s));
  QCD_CUDA(cudaMemcpyAsync(out, d_res, sizeof(double), cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  return QCD_OK;
}

static int gauge_action(qcd_ctx* c, HmcScratch& sc, const double* U, double beta, double* S, cudaStream_t s) {
  const Lex g = lex_of(c);
  const unsigned grid = grid_for(g.V);
  plaquette_kernel<<<grid, kThreads, 0, s>>>(g, (const double2*)U, sc.part);
  QCD_LAUNCHED();
  double sum = 0;
  QCD_TRY(sum_to_host(sc.part, (int)grid, sc.res, &sum, s));
  *S = beta * sum;
  return QCD_OK;
}

static int sumsq(HmcScratch& sc, long long n, const double* v, double* out, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<long long>(grid_for(n), (long long)sc.nparts);
  sumsq_kernel<<<grid, kThreads, 0, s>>>(n, v, sc.part);
  QCD_LAUNCHED();
  return sum_to_host(sc.part, (int)grid, sc.res, out, s);
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_gauge_action(qcd_ctx* c, const double* U, double beta, double* S, void* stream) {
  if (!c || !U || !S) return QCD_ERR_ARG;
  HmcScratch sc;
  QCD_TRY(sc.init(c->V));
  return gauge_action(c, sc, U, beta, S, (cudaStream_t)stream);
}

extern "C" int qcd_gauge_force(qcd_ctx* c, const double* U, double beta, double* F, void* stream) {
  if (!c || !U || !F) return QCD_ERR_ARG;
  const Lex g = lex_of(c);
  gauge_force_kernel<<<grid_for(4 * g.V), kThreads, 0, (cudaStream_t)stream>>>(g, (const double2*)U, beta, F);
  QCD_LAUNCHED();
  return QCD_OK;
}

extern "C" int qcd_update_links(qcd_ctx* c, double* U, const double* pi, double eps, void* stream) {
  if (!c || !U || !pi) return QCD_ERR_ARG;
  const long long n = 4 * c->V;
  link_update_kernel<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(n, (double2*)U, pi, eps);
  QCD_LAUNCHED();
  return QCD_OK;
}

namespace {

struct DevBuf {
  double* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t n) {
    if (cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return QCD_ERR_NOMEM;
    }
    return QCD_OK;
  }
};

// CUDA-event pair timing a region on one stream, released on every exit path
struct EventTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EventTimer() {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  ~EventTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  float elapsed_ms(cudaStream_t s) {
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  }
};

struct Traj {
  qcd_ctx* c;
  cudaStream_t s;
  const qcd_solver_params* sp;
  qcd_hmc_info* info;
  HmcScratch sc;
  DevBuf phi, Y, X, Fg, Ff;
  long long V;

  int load(const double* U) {
    QCD_TRY(qcd_load_gauge(c, U, 1, s));
    return qcd_build_clover(c, s);
  }
  int count(const qcd_solve_info& si) {
    info->solves += 1;
    info->iterations += si.iterations + si.cg_iterations;
    return si.status;
  }
  // Y = D^-+ phi (from zero); returns S_f = |Y|^2
  int fermion_action(double* Sf) {
    QCD_CUDA(cudaMemsetAsync(Y.p, 0, sizeof(double) * 24 * V, s));
    qcd_solve_info si;
    QCD_TRY(qcd_solve_dagger(c, phi.p, Y.p, sp, &si, s));
    QCD_TRY(count(si));
    return sumsq(sc, 24 * V, Y.p, Sf, s);
  }
  int hamiltonian(const double* U, const double* pi, double beta, double* kin, double* Sg, double* Sf) {
    double k2 = 0;
    QCD_TRY(sumsq(sc, 8 * 4 * V, pi, &k2, s));
    *kin = 0.5 * k2;
    QCD_TRY(gauge_action(c, sc, U, beta, Sg, s));
    return fermion_action(Sf);
  }
  // pi -= step (dS_g + dS_f) at the loaded gauge field U
  int momentum_step(const double* U, double* pi, double beta, double step) {
    QCD_TRY(qcd_gauge_force(c, U, beta, Fg.p, s));
    QCD_CUDA(cudaMemsetAsync(Y.p, 0, sizeof(double) * 24 * V, s));
    QCD_CUDA(cudaMemsetAsync(X.p, 0, sizeof(double) * 24 * V, s));
    qcd_solve_info si;
    QCD_TRY(qcd_solve_dagger(c, phi.p, Y.p, sp, &si, s));
    QCD_TRY(count(si));
    QCD_TRY(qcd_solve(c, Y.p, X.p, 1, sp, &si, s));
    QCD_TRY(count(si));
    QCD_TRY(qcd_force(c, X.p, Y.p, Ff.p, s));  // -Re(Y^+ dD X)
    const long long n = 32 * V;
    momentum_update_kernel<<<grid_for(n), kThreads, 0, s>>>(n, pi, Fg.p, Ff.p, 2.0, step);
    QCD_LAUNCHED();
    return QCD_OK;
  }
};

}  // namespace

extern "C" int qcd_hmc_trajectory(qcd_ctx* c, double* U, double* pi, const double* eta, double beta, double eps,
                                  int nsteps, double u_accept, const qcd_solver_params* sp_in, qcd_hmc_info* info,
                                  void* stream) {
  NvtxRange nv("qcd_hmc_trajectory");
  if (!c || !U || !pi || !eta || nsteps < 1 || !(eps > 0)) return QCD_ERR_ARG;
  qcd_hmc_info local;
  if (!info) info = &local;
  memset(info, 0, sizeof(*info));
  qcd_solver_params sp;
  if (sp_in) sp = *sp_in; else qcd_solver_defaults(&sp);
  cudaStream_t s = (cudaStream_t)stream;
  EventTimer timer;
  cudaEventRecord(timer.e0, s);
  Traj t{c, s, &sp, info};
  t.V = c->V;
  const long long V = c->V;
  QCD_TRY(t.sc.init(V));
  DevBuf U0;
  QCD_TRY(U0.alloc(72 * V));
  QCD_TRY(t.phi.alloc(24 * V));
  QCD_TRY(t.Y.alloc(24 * V));
  QCD_TRY(t.X.alloc(24 * V));
  QCD_TRY(t.Fg.alloc(32 * V));
  QCD_TRY(t.Ff.alloc(32 * V));
  QCD_CUDA(cudaMemcpyAsync(U0.p, U, sizeof(double) * 72 * V, cudaMemcpyDeviceToDevice, s));
  // pseudofermion phi = D(U)^+ eta at the start of the trajectory
  QCD_TRY(t.load(U));
  QCD_TRY(qcd_apply_D(c, eta, t.phi.p, 1, QCD_PREC_F64, 1, s));
  QCD_TRY(t.hamiltonian(U, pi, beta, &info->kin0, &info->S_g0, &info->S_f0));
  // leapfrog
  QCD_TRY(t.momentum_step(U, pi, beta, 0.5 * eps));
  for (int k = 0; k < nsteps; ++k) {
    QCD_TRY(qcd_update_links(c, U, pi, eps, s));
    QCD_TRY(t.load(U));
    QCD_TRY(t.momentum_step(U, pi, beta, k < nsteps - 1 ? eps : 0.5 * eps));
  }
  QCD_TRY(t.hamiltonian(U, pi, beta, &info->kin1, &info->S_g1, &info->S_f1));
  info->H0 = info->kin0 + info->S_g0 + info->S_f0;
  info->H1 = info->kin1 + info->S_g1 + info->S_f1;
  info->dH = info->H1 - info->H0;
  info->accepted = (info->dH == info->dH) && u_accept < std::exp(-info->dH);
  if (!info->accepted) {  // restore the starting links (the context keeps the last loaded field)
    QCD_CUDA(cudaMemcpyAsync(U, U0.p, sizeof(double) * 72 * V, cudaMemcpyDeviceToDevice, s));
    QCD_TRY(t.load(U));
  }
  info->time_ms = timer.elapsed_ms(s);
  return QCD_OK;
}
