// Full-lattice clover Wilson-Dirac operator (Sec. 4: the matrix-vector product
// applied to a spinor field; Sec. 6: the double precision operator of the
// outer solver).  One thread per site; the 8 neighbour spinors are gathered
// through L1/L2 (the Schwarz blocks are contiguous and CTAs follow the block
// order, so block faces are re-read from cache, not HBM); links come from the
// site itself (forward hops) and from the backward neighbour.
#include "internal.h"

namespace qcd {

template <int P>
struct Arith {
  typedef float T;
};
template <>
struct Arith<P64> {
  typedef double T;
};

// a neighbour's spinor with its 16-bit scale left out (returned in `scale`,
// 1 for FP32/FP64), so the scale joins the hop coefficient
template <int P, typename T>
__device__ __forceinline__ Spinor<T> load_spinor_unscaled(const FieldPtr& f, int Vb, int blk, int r, T& scale) {
  if constexpr (P == P16 || P == PB16) {
    float v[24];
    scale = load_record_raw<P, 24>(f, Vb, blk, r, v);
    Spinor<T> s;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) s.c[a][b] = {v[6 * a + 2 * b], v[6 * a + 2 * b + 1]};
    return s;
  } else {
    scale = T(1);
    return load_spinor<P, T>(f, Vb, blk, r);
  }
}

// acc += -1/2 [eta U (1 -/+ g) psi(x + mu) + eta U^+ (1 +/- g) psi(x - mu)]; the
// factor -1/2, the boundary sign and the neighbour's 16-bit scale are one
// coefficient per hop (U h is linear in h)
template <int MU, int P, int DAG, typename T>
__device__ __forceinline__ void hop_pair(const Geom& g, const void* U, const FieldPtr& in, int blk, int r,
                                         const int y[4], const int n[4], Spinor<T>& acc) {
  constexpr int SF = DAG ? +1 : -1;  // D: (1 - g) psi(x + mu); D^+: (1 + g) psi(x + mu)
  {
    Nbr f = neighbour(g, blk, y, n, MU, +1);
    T sc;
    Spinor<T> p = load_spinor_unscaled<P, T>(in, g.Vb, f.blk, f.r, sc);
    Half<T> h = project<MU, SF>(p);
    SU3<T> u = load_link<P, T>(U, g.Vb, blk, r, MU);
    Half<T> w = umul(u, h);
    expand_add<MU, SF>(acc, w, (f.wrap ? T(-0.5) * bc_of<T>(g, MU) : T(-0.5)) * sc);
  }
  {
    Nbr b = neighbour(g, blk, y, n, MU, -1);
    T sc;
    Spinor<T> p = load_spinor_unscaled<P, T>(in, g.Vb, b.blk, b.r, sc);
    Half<T> h = project<MU, -SF>(p);
    SU3<T> u = load_link<P, T>(U, g.Vb, b.blk, b.r, MU);
    Half<T> w = udmul(u, h);
    expand_add<MU, -SF>(acc, w, (b.wrap ? T(-0.5) * bc_of<T>(g, MU) : T(-0.5)) * sc);
  }
}

// (D psi)(site) or (D^+ psi)(site); A is Hermitian so D^+ only swaps projectors
template <int P, int DAG, typename T>
__device__ __forceinline__ Spinor<T> dirac_site(const Geom& g, const void* U, const FieldPtr& A, const FieldPtr& in,
                                               int blk, int r) {
  int n[4], y[4];
  block_coords(g, blk, n);
  const int packed = __ldg(g.r2y + r);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) y[mu] = ycoord(packed, mu);
  Spinor<T> acc;
  zero(acc);
  hop_pair<0, P, DAG, T>(g, U, in, blk, r, y, n, acc);
  hop_pair<1, P, DAG, T>(g, U, in, blk, r, y, n, acc);
  hop_pair<2, P, DAG, T>(g, U, in, blk, r, y, n, acc);
  hop_pair<3, P, DAG, T>(g, U, in, blk, r, y, n, acc);
  T sp;
  Spinor<T> psi = load_spinor_unscaled<P, T>(in, g.Vb, blk, r, sp);
  if constexpr (P == P16 || P == PB16) {
    // one chiral 6x6 block at a time: chunks 4 hb .. 4 hb + 4 hold its 18
    // packed pairs from pair 2 hb on
    const uint4* d = (const uint4*)A.data + (long long)blk * 9 * g.Vb + r;
    const T s = (A.norm ? __ldg(A.norm + (long long)blk * g.Vb + r) : 1.0f) * sp;
#pragma unroll
    for (int hb = 0; hb < 2; ++hb) {
      uint32_t w[20];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const uint4 v = __ldg(d + (long long)(4 * hb + k) * g.Vb);
        w[4 * k] = v.x;
        w[4 * k + 1] = v.y;
        w[4 * k + 2] = v.z;
        w[4 * k + 3] = v.w;
      }
      T c[36];
#pragma unroll
      for (int k = 0; k < 18; ++k) {
        const float2 x = to_f2<P>(w[2 * hb + k]);
        c[2 * k] = x.x;
        c[2 * k + 1] = x.y;
      }
      cpx<T> i6[6], o6[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) i6[i] = psi.c[2 * hb + i / 3][i % 3];
      clover_block_apply(c, i6, o6);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        cpx<T>& a = acc.c[2 * hb + i / 3][i % 3];
        a = {fma(s, o6[i].re, a.re), fma(s, o6[i].im, a.im)};
      }
    }
  } else {
    T c[72];
    load_record<P, 72, T>(A, g.Vb, blk, r, c);
    const Spinor<T> o = clover_apply(c, psi);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) acc.c[a][b] = acc.c[a][b] + o.c[a][b];
  }
  return acc;
}

// Schwarz block shapes with their own instantiation: BS = 1 for 4^4 and 2 for
// 8 x 4^3 (time extent 8); the in-block extents, strides and volume are then
// compile-time constants, which shortens the neighbour and address arithmetic
static int block_shape_id(const Geom& g) {
  if (g.b[1] == 4 && g.b[2] == 4 && g.b[3] == 4) {
    if (g.b[0] == 4) return 1;
    if (g.b[0] == 8) return 2;
  }
  return 0;
}

template <int BS>
__device__ __forceinline__ void fix_block_shape(Geom& g) {
  if constexpr (BS != 0) {
    constexpr int b0 = BS == 1 ? 4 : 8;
    g.b[0] = b0;
    g.b[1] = g.b[2] = g.b[3] = 4;
    g.ystr[0] = 64;
    g.ystr[1] = 16;
    g.ystr[2] = 4;
    g.ystr[3] = 1;
    g.Vb = 64 * b0;
    g.Vbh = 32 * b0;
  }
}

// one thread per site; with nrhs > 1 the thread applies the operator to every
// right-hand side in turn (fields nrhs apart by `stride` sites), so the
// site's links and clover block come from HBM once and from L1 afterwards.
// The FP32 instantiation is told it runs one 512-thread CTA per SM (the full
// 128 registers, used to issue more gathers ahead); the others keep the
// compiler's default
template <int P, int DAG, int BS>
__global__ void __launch_bounds__(512, P == P32 ? 1 : 0) dirac_kernel(Geom g0, const void* __restrict__ U, FieldPtr A, FieldPtr in,
                                                    FieldPtr out, int nrhs) {
  typedef typename Arith<P>::T T;
  Geom g = g0;
  fix_block_shape<BS>(g);
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  constexpr int NC = P == P64 ? 12 : (P == P32 ? 6 : 3);
#pragma unroll 1
  for (int k = 0; k < nrhs; ++k) {
    FieldPtr fi = in, fo = out;
    fi.data = (char*)in.data + (size_t)k * g.V * NC * 16;
    fo.data = (char*)out.data + (size_t)k * g.V * NC * 16;
    if (in.norm) fi.norm = in.norm + (size_t)k * g.V;
    if (out.norm) fo.norm = out.norm + (size_t)k * g.V;
    Spinor<T> o = dirac_site<P, DAG, T>(g, U, A, fi, blk, r);
    store_spinor<P, T>(fo, g.Vb, blk, r, o);
  }
}

// deterministic block sum of a double: warp shuffles, then warps in order
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;
}

// r = b - D x (FP64), partial[blockIdx.x] = sum |r|^2 over the CTA
__global__ void __launch_bounds__(256) residual64_kernel(Geom g, const void* __restrict__ U, FieldPtr A, FieldPtr b,
                                                         FieldPtr x, FieldPtr r_out, double* partial) {
  __shared__ double sh[32];
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double nrm = 0;
  if (s < g.V) {
    int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
    Spinor<double> o = dirac_site<P64, 0, double>(g, U, A, x, blk, r);
    Spinor<double> bb = load_spinor<P64, double>(b, g.Vb, blk, r);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        o.c[sp][a] = bb.c[sp][a] - o.c[sp][a];
        nrm += o.c[sp][a].re * o.c[sp][a].re + o.c[sp][a].im * o.c[sp][a].im;
      }
    store_spinor<P64, double>(r_out, g.Vb, blk, r, o);
  }
  double t = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

static double bytes_per_site(int prec) {
  if (prec == P64) return 2 * 24 * 8 + 4 * 18 * 8 + 72 * 8;
  if (prec == P32) return 2 * 24 * 4 + 4 * 12 * 4 + 72 * 4;
  return 2 * (24 * 2 + 4) + 4 * 12 * 2 + (72 * 2 + 4);
}

int dirac_apply(qcd_ctx* c, const Rec& in, const Rec& out, int dagger, cudaStream_t s, int nrhs) {
  const int prec = in.prec;
  if (out.prec != prec || in.nreal != 24 || out.nreal != 24 || nrhs < 1) return QCD_ERR_ARG;
  QCD_TRY(ensure_gauge(c, prec, s));
  QCD_TRY(ensure_clover(c, prec, s));
  const int threads = c->dirac_threads[prec];
  const unsigned grid = (unsigned)((c->V + threads - 1) / threads);
  const void* U = c->U[prec];
  FieldPtr A = c->A[prec].ptr();
  // algorithmic bytes: links and clover once, spinors per right-hand side
  const double spin = prec == P64 ? 384 : (prec == P32 ? 192 : 104);
  const double bytes = ((bytes_per_site(prec) - spin) + spin * nrhs) * (double)c->V;
  ProfScope ps(c, QCD_KERNEL_DIRAC, s, bytes, 1824.0 * (double)c->V * nrhs);
#define LAUNCH(PP, BS)                                                                                 \
  if (dagger)                                                                                          \
    dirac_kernel<PP, 1, BS><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs);           \
  else                                                                                                 \
    dirac_kernel<PP, 0, BS><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs);
  // 16-bit storage (FP16, BF16) is issue-bound, so it gets the fixed-shape instantiations
  const int bs = block_shape_id(c->g);
  switch (prec) {
    case P64: LAUNCH(P64, 0); break;
    case P32: LAUNCH(P32, 0); break;
    case P16:
      if (bs == 1) {
        LAUNCH(P16, 1);
      } else if (bs == 2) {
        LAUNCH(P16, 2);
      } else {
        LAUNCH(P16, 0);
      }
      break;
    case PB16:
      if (bs == 1) {
        LAUNCH(PB16, 1);
      } else if (bs == 2) {
        LAUNCH(PB16, 2);
      } else {
        LAUNCH(PB16, 0);
      }
      break;
    default: return QCD_ERR_ARG;
  }
#undef LAUNCH
  QCD_LAUNCHED();
  return QCD_OK;
}

int residual64(qcd_ctx* c, double* part, const Rec& b, const Rec& x, const Rec& r, double* d_norm2, cudaStream_t s) {
  NvtxRange nv("residual64");
  if (b.prec != P64 || x.prec != P64 || r.prec != P64) return QCD_ERR_ARG;
  QCD_TRY(ensure_gauge(c, P64, s));
  QCD_TRY(ensure_clover(c, P64, s));
  const unsigned grid = (unsigned)((c->V + 255) / 256);
  {
    ProfScope ps(c, QCD_KERNEL_RESIDUAL, s, (bytes_per_site(P64) + 192) * (double)c->V, 1848.0 * (double)c->V);
    residual64_kernel<<<grid, 256, 0, s>>>(c->g, c->U[P64], c->A[P64].ptr(), b.ptr(), x.ptr(), r.ptr(),
                                           part);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_norm2, s);
}

// ------------------------------------------------------------------------
// Even/odd split of D over the whole lattice (the global parity of a site is
// its block-local parity, block extents being even).  For the sites of
// parity `par` (r = par * Vbh + rr):
//   PRE = 1:  out = c1 * M x + c2 * H y
//   PRE = 0:  out = M (c1 x + c2 H y)
// with H y = -1/2 sum of the hops from the opposite parity (D's hopping term,
// its adjoint's with DAG), M = Ahat on these sites (A_ee on even, A_oo^-1 on
// odd) if USE_M, else 1.  x and out are read / written on parity par only, y
// on the other parity only, so out may be y.  c2 = 0 skips the hops, c1 = 0
// the load of x.  FP64 throughout.
// ------------------------------------------------------------------------
template <int DAG, int PRE, int USE_M>
__global__ void __launch_bounds__(256, 2) eo_kernel(Geom g, const void* __restrict__ U, FieldPtr Ahat, FieldPtr x,
                                                 FieldPtr y, FieldPtr out, int par, double c1, double c2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.V / 2) return;
  const int blk = (int)(t / g.Vbh), r = (int)(t - (long long)blk * g.Vbh) + par * g.Vbh;
  Spinor<double> h;
  zero(h);
  if (c2 != 0.0) {
    int n[4], yc[4];
    block_coords(g, blk, n);
    const int packed = __ldg(g.r2y + r);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) yc[mu] = ycoord(packed, mu);
    hop_pair<0, P64, DAG, double>(g, U, y, blk, r, yc, n, h);
    hop_pair<1, P64, DAG, double>(g, U, y, blk, r, yc, n, h);
    hop_pair<2, P64, DAG, double>(g, U, y, blk, r, yc, n, h);
    hop_pair<3, P64, DAG, double>(g, U, y, blk, r, yc, n, h);
  }
  Spinor<double> v;
  zero(v);
  if (c1 != 0.0) v = load_spinor<P64, double>(x, g.Vb, blk, r);
  double cm[72];
  if (USE_M) load_record<P64, 72, double>(Ahat, g.Vb, blk, r, cm);
  if (PRE && USE_M) v = clover_apply(cm, v);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      v.c[a][b] = {fma(c2, h.c[a][b].re, c1 * v.c[a][b].re), fma(c2, h.c[a][b].im, c1 * v.c[a][b].im)};
  if (!PRE && USE_M) v = clover_apply(cm, v);
  store_spinor<P64, double>(out, g.Vb, blk, r, v);
}

int eo_apply(qcd_ctx* c, const Rec& x, const Rec& y, const Rec& out, int par, int dagger, int pre, int use_m,
             double c1, double c2, cudaStream_t s) {
  if (x.prec != P64 || y.prec != P64 || out.prec != P64 || (par != 0 && par != 1)) return QCD_ERR_ARG;
  QCD_TRY(ensure_gauge(c, P64, s));
  QCD_TRY(ensure_clover(c, P64, s));
  const unsigned grid = (unsigned)((c->V / 2 + 255) / 256);
  // algorithmic bytes: per site of parity par, 8 neighbour spinors and 8 links
  // (hops), x and the clover record (if used) and the result
  const double sites = (double)c->V / 2;
  const double bytes = sites * ((c2 != 0.0 ? 8 * 192 + 8 * 144 : 0) + (c1 != 0.0 ? 192 : 0) + (use_m ? 576 : 0) + 192);
  ProfScope ps(c, QCD_KERNEL_DIRAC, s, bytes, sites * ((c2 != 0.0 ? 1320.0 : 0.0) + (use_m ? 504.0 : 0.0)));
  const void* U = c->U[P64];
  const FieldPtr A = c->Ahat[P64].ptr();
#define EO(D, P, M) eo_kernel<D, P, M><<<grid, 256, 0, s>>>(c->g, U, A, x.ptr(), y.ptr(), out.ptr(), par, c1, c2)
  if (dagger) {
    if (pre) { if (use_m) EO(1, 1, 1); else EO(1, 1, 0); }
    else { if (use_m) EO(1, 0, 1); else EO(1, 0, 0); }
  } else {
    if (pre) { if (use_m) EO(0, 1, 1); else EO(0, 1, 0); }
    else { if (use_m) EO(0, 0, 1); else EO(0, 0, 0); }
  }
#undef EO
  QCD_LAUNCHED();
  return QCD_OK;
}

// out_e = Dhat x_e = A_ee x_e - H_eo A_oo^-1 H_oe x_e (dagger: Dhat^+, the same
// with the adjoint's hops); tmp receives A_oo^-1 H_oe x_e on the odd sites.
// Only the even sites of x and out are read / written.
int schur_apply(qcd_ctx* c, const Rec& x, const Rec& tmp, const Rec& out, int dagger, cudaStream_t s) {
  QCD_TRY(eo_apply(c, x, x, tmp, 1, dagger, 0, 1, 0.0, 1.0, s));
  return eo_apply(c, x, tmp, out, 0, dagger, 1, 1, 1.0, -1.0, s);
}

}  // namespace qcd
