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
                                                    FieldPtr out, int nrhs, const int* __restrict__ mask,
                                                    int out_df) {
  typedef typename Arith<P>::T T;
  Geom g = g0;
  fix_block_shape<BS>(g);
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  constexpr int NC = P == P64 ? 12 : (P == P32 ? 6 : 3);
#pragma unroll 1
  for (int k = 0; k < nrhs; ++k) {
    if (mask && !mask[k]) continue;  // a right-hand side of a batch that is not being iterated
    FieldPtr fi = in, fo = out;
    fi.data = (char*)in.data + (size_t)k * g.V * NC * 16;
    fo.data = (char*)out.data + (size_t)k * g.V * NC * 16;
    if (in.norm) fi.norm = in.norm + (size_t)k * g.V;
    if (out.norm) fo.norm = out.norm + (size_t)k * g.V;
    Spinor<T> o = dirac_site<P, DAG, T>(g, U, A, fi, blk, r);
    if constexpr (P == P64) {
      if (out_df) {  // the FP64 result split into double-float pairs for a df64 recursion
        store_spinor<PDF, T>(fo, g.Vb, blk, r, o);
        continue;
      }
    }
    store_spinor<P, T>(fo, g.Vb, blk, r, o);
  }
}

// ------------------------------------------------------------------------
// Two threads per site (16-bit storage).  The one-thread form above needs all
// 128 registers for a site's eight hops, which leaves 16 warps per SM to hide
// the gathers.  Here thread half hf of a CTA (warp-uniform: threads
// hf * 128 .. hf * 128 + 127) computes the hops in directions 2 hf and
// 2 hf + 1 of 128 sites and owns spin components 2 hf, 2 hf + 1 of their
// results: the partial hop sums of the other two components go to the partner
// through shared memory (a named barrier of the two warps that hold the same
// 32 sites), the clover term acts on the owned chiral half alone (it is block
// diagonal in chirality), and the per-site 16-bit scale of the result is the
// larger of the two halves' maxima.
// ------------------------------------------------------------------------
static constexpr int kPairSites = 128;  // sites per CTA of the two-thread form (256 threads)
// resident CTAs per SM the two-thread form is compiled for (its register budget)
#ifndef QCD_PAIR_MIN_CTAS
#define QCD_PAIR_MIN_CTAS 2
#endif

// owned half (spins 2 hf, 2 hf + 1) of a 16-bit spinor record without its scale
// (16-bit words 6 hf .. 6 hf + 5: chunk 2 hf and the hf-th 8-byte half of chunk 1)
template <int P>
__device__ __forceinline__ Half<float> load_half16_unscaled(const FieldPtr& f, int Vb, int blk, int r, int hf) {
  const uint4* d = (const uint4*)f.data + (long long)blk * 3 * Vb + r;
  const uint4 a = __ldg(d + (long long)(2 * hf) * Vb);
  const uint2 b = __ldg((const uint2*)(d + Vb) + hf);
  const uint32_t w[6] = {hf ? b.x : a.x, hf ? b.y : a.y, hf ? a.x : a.z, hf ? a.y : a.w, hf ? a.z : b.x, hf ? a.w : b.y};
  Half<float> h;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 x = to_f2<P>(w[k]);
    h.c[k / 3][k % 3] = {x.x, x.y};
  }
  return h;
}

// store the owned half with the site's scale (the maximum over both halves)
template <int P>
__device__ __forceinline__ void store_half16(const FieldPtr& f, int Vb, int blk, int r, int hf, const Half<float>& h,
                                             float scale) {
  typedef typename Storage<P>::real hr;
  const float inv = scale > 0.f ? 1.0f / scale : 0.f;
  uint32_t w[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    hr* q = reinterpret_cast<hr*>(&w[k]);
    q[0] = from_f<P>(h.c[k / 3][k % 3].re * inv);
    q[1] = from_f<P>(h.c[k / 3][k % 3].im * inv);
  }
  uint4* d = (uint4*)f.data + (long long)blk * 3 * Vb + r;
  if (hf == 0) {
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    *((uint2*)(d + Vb)) = make_uint2(w[4], w[5]);
    f.norm[(long long)blk * Vb + r] = scale;
  } else {
    *((uint2*)(d + Vb) + 1) = make_uint2(w[0], w[1]);
    d[2 * (long long)Vb] = make_uint4(w[2], w[3], w[4], w[5]);
  }
}

template <int P, int DAG, int BS>
__global__ void __launch_bounds__(2 * kPairSites, QCD_PAIR_MIN_CTAS) dirac_pair_kernel(Geom g0, const void* __restrict__ U, FieldPtr A,
                                                                  FieldPtr in, FieldPtr out, int nrhs,
                                                                  const int* __restrict__ mask) {
  static_assert(P == P16 || P == PB16, "16-bit storage only");
  __shared__ float xch[2][12][kPairSites];  // [receiving half][real][site]
  __shared__ float mx[2][kPairSites];
  Geom g = g0;
  fix_block_shape<BS>(g);
  const int hf = threadIdx.x / kPairSites, li = threadIdx.x - hf * kPairSites;
  const long long s = (long long)blockIdx.x * kPairSites + li;
  const bool act = s < g.V;
  const long long sc = act ? s : 0;
  const int blk = (int)(sc / g.Vb), r = (int)(sc - (long long)blk * g.Vb);
  int n[4], y[4];
  block_coords(g, blk, n);
  {
    const int packed = __ldg(g.r2y + r);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) y[mu] = ycoord(packed, mu);
  }
  const int pair_bar = 1 + (li >> 5);  // named barrier of warps li / 32 and li / 32 + 4
#pragma unroll 1
  for (int k = 0; k < nrhs; ++k) {
    if (mask && !mask[k]) continue;
    FieldPtr fi = in, fo = out;
    fi.data = (char*)in.data + (size_t)k * g.V * 3 * 16;
    fo.data = (char*)out.data + (size_t)k * g.V * 3 * 16;
    fi.norm = in.norm + (size_t)k * g.V;
    fo.norm = out.norm + (size_t)k * g.V;
    Spinor<float> acc;
    zero(acc);
    if (hf) {
      hop_pair<2, P, DAG, float>(g, U, fi, blk, r, y, n, acc);
      hop_pair<3, P, DAG, float>(g, U, fi, blk, r, y, n, acc);
    } else {
      hop_pair<0, P, DAG, float>(g, U, fi, blk, r, y, n, acc);
      hop_pair<1, P, DAG, float>(g, U, fi, blk, r, y, n, acc);
    }
    // hand the partner its components
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cpx<float> v = acc.c[2 * (1 - hf) + sp][c];
        xch[1 - hf][6 * sp + 2 * c][li] = v.re;
        xch[1 - hf][6 * sp + 2 * c + 1][li] = v.im;
      }
    asm volatile("bar.sync %0, 64;" ::"r"(pair_bar) : "memory");
    Half<float> o;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        o.c[sp][c] = {acc.c[2 * hf + sp][c].re + xch[hf][6 * sp + 2 * c][li],
                      acc.c[2 * hf + sp][c].im + xch[hf][6 * sp + 2 * c + 1][li]};
    // clover: chiral block hf on the site's own half
    {
      const Half<float> psi = load_half16_unscaled<P>(fi, g.Vb, blk, r, hf);
      const float ps = __ldg(fi.norm + (long long)blk * g.Vb + r);
      const uint4* d = (const uint4*)A.data + (long long)blk * 9 * g.Vb + r;
      const float scl = (A.norm ? __ldg(A.norm + (long long)blk * g.Vb + r) : 1.0f) * ps;
      uint32_t w[20];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const uint4 v = __ldg(d + (long long)(4 * hf + q) * g.Vb);
        w[4 * q] = v.x;
        w[4 * q + 1] = v.y;
        w[4 * q + 2] = v.z;
        w[4 * q + 3] = v.w;
      }
      float cb[36];
#pragma unroll
      for (int q = 0; q < 18; ++q) {
        const float2 x = to_f2<P>(hf ? w[q + 2] : w[q]);
        cb[2 * q] = x.x;
        cb[2 * q + 1] = x.y;
      }
      cpx<float> i6[6], o6[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) i6[q] = psi.c[q / 3][q % 3];
      clover_block_apply(cb, i6, o6);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        cpx<float>& a = o.c[q / 3][q % 3];
        a = {fmaf(scl, o6[q].re, a.re), fmaf(scl, o6[q].im, a.im)};
      }
    }
    float m = 0.f;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) m = fmaxf(m, fmaxf(fabsf(o.c[sp][c].re), fabsf(o.c[sp][c].im)));
    mx[hf][li] = m;
    asm volatile("bar.sync %0, 64;" ::"r"(pair_bar) : "memory");
    m = fmaxf(m, mx[1 - hf][li]);
    if (act) store_half16<P>(fo, g.Vb, blk, r, hf, o, m);
  }
}

// ------------------------------------------------------------------------
// The operator in double-float arithmetic: spinors, links (all 18 reals) and
// clover as (hi, lo) pairs of FP32 values (the FP64 layouts with float4 =
// (re hi, re lo, im hi, im lo) per complex number), computed on the FP32
// units with error-free transformations.  Every output real is a double-float
// running sum (dfacc); a hop's projection adds pairs by TwoSum, its SU(3)
// product accumulates exact FP32 products and their cross terms, its
// expansion and the -1/2 (a power of two) are exact.  About 12 FP32 operations
// per real multiply-add in place of one FP64 fused multiply-add, on units 64
// times faster on GB300; the result agrees with the FP64 operator to about
// 2^-46 relative.
// ------------------------------------------------------------------------
struct cdf {
  df re, im;
};
__device__ __forceinline__ cdf cdf_of(const float4& v) { return {{v.x, v.y}, {v.z, v.w}}; }
// x + y without the final renormalisation (a valid double-float operand)
__device__ __forceinline__ df dsum(df x, df y) {
  df t = two_sum(x.hi, y.hi);
  t.lo += x.lo + y.lo;
  return t;
}
__device__ __forceinline__ cdf cplus(const cdf& x, const cdf& y) { return {dsum(x.re, y.re), dsum(x.im, y.im)}; }
__device__ __forceinline__ cdf cminus(const cdf& x, const cdf& y) {
  return {dsum(x.re, df_neg(y.re)), dsum(x.im, df_neg(y.im))};
}
__device__ __forceinline__ cdf ctimes_i(const cdf& z) { return {df_neg(z.im), z.re}; }   // i z
__device__ __forceinline__ cdf ctimes_mi(const cdf& z) { return {z.im, df_neg(z.re)}; }  // -i z

// (ar, ai) += u h and (ar, ai) += conj(u) h
__device__ __forceinline__ void cmac_df(dfacc& ar, dfacc& ai, const cdf& u, const cdf& h) {
  acc_prod(ar, u.re.hi, u.re.lo, h.re.hi, h.re.lo);
  acc_prod(ar, -u.im.hi, -u.im.lo, h.im.hi, h.im.lo);
  acc_prod(ai, u.re.hi, u.re.lo, h.im.hi, h.im.lo);
  acc_prod(ai, u.im.hi, u.im.lo, h.re.hi, h.re.lo);
}
__device__ __forceinline__ void cjmac_df(dfacc& ar, dfacc& ai, const cdf& u, const cdf& h) {
  acc_prod(ar, u.re.hi, u.re.lo, h.re.hi, h.re.lo);
  acc_prod(ar, u.im.hi, u.im.lo, h.im.hi, h.im.lo);
  acc_prod(ai, u.re.hi, u.re.lo, h.im.hi, h.im.lo);
  acc_prod(ai, -u.im.hi, -u.im.lo, h.re.hi, h.re.lo);
}

struct SpinAcc {
  dfacc re[4][3], im[4][3];
};

// acc[s][c] += f z for f = +-1/2 (exact) and a lazily summed z = (zr, zi)
__device__ __forceinline__ void acc_cadd(SpinAcc& a, int s, int c, float f, const dfacc& zr, const dfacc& zi) {
  acc_add(a.re[s][c], f * zr.s, f * zr.c);
  acc_add(a.im[s][c], f * zi.s, f * zi.c);
}
// acc[s][c] += f i z
__device__ __forceinline__ void acc_cadd_i(SpinAcc& a, int s, int c, float f, const dfacc& zr, const dfacc& zi) {
  acc_add(a.re[s][c], -f * zi.s, -f * zi.c);
  acc_add(a.im[s][c], f * zr.s, f * zr.c);
}

// z times a phase +-1 or +-i: (im ? i z : z) * sg
__device__ __forceinline__ cdf cphase(const cdf& z, bool im, float sg) {
  const df re = im ? df_neg(z.im) : z.re, imv = im ? z.re : z.im;
  return {{sg * re.hi, sg * re.lo}, {sg * imv.hi, sg * imv.lo}};
}

// The eight hops share one loop body (direction, projection sign and link
// conjugation chosen at run time), and the two clover blocks another: the
// double-float arithmetic is long, and unrolled over every hop it would not
// fit the instruction cache.
// what a double-float hop needs to find its neighbour: the site's in-block
// lexicographic index, its packed local coordinates (8 bits each), its block
// coordinates (16 bits each) and its parity; kept in five registers (a table
// of the eight neighbours would take 24 and make the kernel spill), the
// neighbours are computed per hop
struct DfSite {
  int j, py, pn01, pn23, par;
};

__device__ __forceinline__ DfSite df_site_info(const Geom& g, int blk, int r) {
  int n[4];
  block_coords(g, blk, n);
  DfSite d;
  d.py = __ldg(g.r2y + r);
  d.pn01 = n[0] | (n[1] << 16);
  d.pn23 = n[2] | (n[3] << 16);
  d.j = 0;
  d.par = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    d.j += ycoord(d.py, mu) * g.ystr[mu];
    d.par += ycoord(d.py, mu);
  }
  d.par &= 1;
  return d;
}

// neighbour of hop h (mu = h / 2, forward for even h): block, site and the
// hop's coefficient -1/2 (times the boundary sign where it wraps around)
__device__ __forceinline__ void df_hop_nbr(const Geom& g, int blk, const DfSite& d, int h, int& hb, int& hr,
                                           float& cf) {
  const int mu = h >> 1;
  const int ymu = ycoord(d.py, mu), nmu = ((mu < 2 ? d.pn01 : d.pn23) >> (16 * (mu & 1))) & 0xffff;
  const int b = g.b[mu], ys = g.ystr[mu], nb = g.nb[mu], bs = g.bstr[mu];
  int j = d.j;
  bool wrap = false;
  hb = blk;
  if ((h & 1) == 0) {
    if (ymu + 1 < b) {
      j += ys;
    } else {
      j -= (b - 1) * ys;
      wrap = nmu + 1 == nb;
      hb += wrap ? -(nb - 1) * bs : bs;
    }
  } else {
    if (ymu > 0) {
      j -= ys;
    } else {
      j += (b - 1) * ys;
      wrap = nmu == 0;
      hb += wrap ? (nb - 1) * bs : -bs;
    }
  }
  hr = (d.par ^ 1) * g.Vbh + (j >> 1);  // even block extents: rank among the parity is j >> 1
  cf = wrap ? -0.5f * g.bcf[mu] : -0.5f;
}

// complex q (= 3 spin + colour) of site (blk, r) of a spinor field as a
// double-float pair: from a double-float field (chunk q holds re hi, re lo, im
// hi, im lo) or, IN32, from an FP32 field (chunk q / 2 holds complexes 2 (q / 2)
// and 2 (q / 2) + 1; the low parts are 0)
template <bool IN32>
__device__ __forceinline__ cdf df_load(const float4* __restrict__ f, int Vb, int blk, int r, int q) {
  if constexpr (IN32) {
    const float2 v = __ldg((const float2*)(f + ((long long)blk * 6 + (q >> 1)) * Vb + r) + (q & 1));
    return cdf{df{v.x, 0.f}, df{v.y, 0.f}};
  } else {
    return cdf_of(__ldg(f + ((long long)blk * 12 + q) * Vb + r));
  }
}

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// the lines hop h reads (the neighbour's spinor and the link) asked for in L1
// one hop ahead: the arithmetic of a hop is long, and the gathers of the next
// one then find their lines near instead of waiting a DRAM round trip
template <bool IN32>
__device__ __forceinline__ void df_prefetch_hop(const Geom& g, const float4* __restrict__ U,
                                                const float4* __restrict__ fin, int blk, int r, const DfSite& ds,
                                                int h) {
  int hb, hr;
  float cf;
  df_hop_nbr(g, blk, ds, h, hb, hr, cf);
  constexpr int NQ = IN32 ? 6 : 12;
#pragma unroll
  for (int q = 0; q < NQ; ++q) prefetch_l1(fin + ((long long)hb * NQ + q) * g.Vb + hr);
  const int mu = h >> 1, bwd = h & 1;
  const float4* ud = U + ((long long)((bwd ? hb : blk) * 4 + mu) * 9) * g.Vb + (bwd ? hr : r);
#pragma unroll
  for (int k = 0; k < 9; ++k) prefetch_l1(ud + (long long)k * g.Vb);
}

// (D psi)(x) (D^+ with DAG) at site (blk, r) of the field fin (double-float,
// or FP32 with IN32), into the double-float accumulators acc
template <int DAG, bool IN32 = false>
__device__ __forceinline__ void df_site(const Geom& g, const float4* __restrict__ U, const FieldPtr& A,
                                        const float4* __restrict__ fin, int blk, int r, const DfSite& ds,
                                        SpinAcc& acc) {
  constexpr float SF = DAG ? 1.f : -1.f;  // D: (1 - g) psi(x + mu); D^+: (1 + g) psi(x + mu)
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.re[sp][c] = acc.im[sp][c] = dfacc{0.f, 0.f};
#pragma unroll 1
  for (int h = 0; h < 8; ++h) {
    const int mu = h >> 1, bwd = h & 1;
    int hb, hr;
    float cf;
    df_hop_nbr(g, blk, ds, h, hb, hr, cf);
    if (h < 7) df_prefetch_hop<IN32>(g, U, fin, blk, r, ds, h + 1);
    // chiral-basis projection (1 + S g_mu): h_i = p_i + S ph_i p_{sigma_i}, with
    // sigma = (2, 3) or (3, 2) and phases -1 / -i (see SpinDir)
    const bool swap = mu == 1 || mu == 2;
    const bool im0 = mu == 1 || mu == 3, im1 = im0;
    const float sg0 = -1.f, sg1 = (mu >= 2) ? 1.f : -1.f;
    const float S = bwd ? -SF : SF;
    cdf hh[2][3];
    {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const cdf p0 = df_load<IN32>(fin, g.Vb, hb, hr, a), p1 = df_load<IN32>(fin, g.Vb, hb, hr, 3 + a);
        const cdf p2 = df_load<IN32>(fin, g.Vb, hb, hr, 6 + a), p3 = df_load<IN32>(fin, g.Vb, hb, hr, 9 + a);
        hh[0][a] = cplus(p0, cphase(swap ? p3 : p2, im0, S * sg0));
        hh[1][a] = cplus(p1, cphase(swap ? p2 : p3, im1, S * sg1));
      }
    }
    // w = U h (forward, the site's link) or U^+ h (backward, the neighbour's link)
    const float4* ud = U + ((long long)((bwd ? hb : blk) * 4 + mu) * 9) * g.Vb + (bwd ? hr : r);
    const float cj = bwd ? -1.f : 1.f;
    dfacc wr[2][3], wi[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) wr[sp][a] = wi[sp][a] = dfacc{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        cdf u = cdf_of(__ldg(ud + (long long)(bwd ? 3 * b + a : 3 * a + b) * g.Vb));
        u.im = {cj * u.im.hi, cj * u.im.lo};
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) cmac_df(wr[sp][a], wi[sp][a], u, hh[sp][b]);
      }
    // acc += cf [w ; S B^+ w]: B^+ w has components conj(ph_i) w_i on spins sigma_i
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc_cadd(acc, 0, a, cf, wr[0][a], wi[0][a]);
      acc_cadd(acc, 1, a, cf, wr[1][a], wi[1][a]);
      // l_i = S cf conj(ph_i) w_i: conj of a real phase is itself, of -i is +i
      const float f0 = S * cf * (im0 ? -sg0 : sg0), f1 = S * cf * (im1 ? -sg1 : sg1);
      dfacc l0r = wr[0][a], l0i = wi[0][a], l1r = wr[1][a], l1i = wi[1][a];
      if (im0) {  // times i: (re, im) -> (-im, re)
        l0r = {-wi[0][a].s, -wi[0][a].c};
        l0i = wr[0][a];
        l1r = {-wi[1][a].s, -wi[1][a].c};
        l1i = wr[1][a];
      }
      acc_cadd(acc, 2, a, swap ? f1 : f0, swap ? l1r : l0r, swap ? l1i : l0i);
      acc_cadd(acc, 3, a, swap ? f0 : f1, swap ? l0r : l1r, swap ? l0i : l1i);
    }
  }
  // clover: two Hermitian 6x6 chiral blocks (6 diagonal reals, then the 15
  // upper off-diagonal elements), record chunk 18 hb + j = reals 36 hb + 2 j, + 1
  const float4* ca = (const float4*)A.data + (long long)blk * 36 * g.Vb + r;
#pragma unroll 1
  for (int hb = 0; hb < 2; ++hb) {
    cdf psi[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) psi[i] = df_load<IN32>(fin, g.Vb, blk, r, 6 * hb + i);
    dfacc tr[6], ti[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) tr[i] = ti[i] = dfacc{0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 6; i += 2) {  // diagonal reals i, i + 1
      const float4 dv = __ldg(ca + (long long)(18 * hb + i / 2) * g.Vb);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int ii = i + q;
        const float dh = q ? dv.z : dv.x, dl = q ? dv.w : dv.y;
        acc_prod(tr[ii], dh, dl, psi[ii].re.hi, psi[ii].re.lo);
        acc_prod(ti[ii], dh, dl, psi[ii].im.hi, psi[ii].im.lo);
      }
    }
    int kk = 3;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        const cdf a = cdf_of(__ldg(ca + (long long)(18 * hb + kk) * g.Vb));
        ++kk;
        cmac_df(tr[i], ti[i], a, psi[j]);
        cjmac_df(tr[j], ti[j], a, psi[i]);
      }
    // into spins 2 hb, 2 hb + 1
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (hb == 0) {
        acc_add(acc.re[i / 3][i % 3], tr[i].s, tr[i].c);
        acc_add(acc.im[i / 3][i % 3], ti[i].s, ti[i].c);
      } else {
        acc_add(acc.re[2 + i / 3][i % 3], tr[i].s, tr[i].c);
        acc_add(acc.im[2 + i / 3][i % 3], ti[i].s, ti[i].c);
      }
    }
  }
}

//
// IN32: the input is an FP32 field (an FP32-exact operand, e.g. a preconditioner
// output), read at half the bytes; the arithmetic is the same
template <int DAG, bool IN32>
__global__ void __launch_bounds__(256, 2) dirac_df_kernel(Geom g, const float4* __restrict__ U, FieldPtr A,
                                                          FieldPtr in, FieldPtr out, int nrhs,
                                                          const int* __restrict__ mask) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  const DfSite ds = df_site_info(g, blk, r);
#pragma unroll 1
  for (int k = 0; k < nrhs; ++k) {
    if (mask && !mask[k]) continue;
    const float4* fin = (const float4*)in.data + (size_t)k * g.V * (IN32 ? 6 : 12);
    float4* fout = (float4*)out.data + (size_t)k * g.V * 12;
    SpinAcc acc;
    df_site<DAG, IN32>(g, U, A, fin, blk, r, ds, acc);
    float4* o = fout + (long long)blk * 12 * g.Vb + r;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const df re = acc_df(acc.re[q / 3][q % 3]), im = acc_df(acc.im[q / 3][q % 3]);
      o[(long long)q * g.Vb] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
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

// r = b - D x with x given as its double-float split: D x in double-float
// arithmetic (as dirac_df_kernel), the difference and |r|^2 in FP64;
// partial[blockIdx.x] = sum |r|^2 over the CTA, blockIdx.y a right-hand side
// of a batch (fields V sites apart, partial sums ps doubles apart)
__global__ void __launch_bounds__(256, 2) residual_df_kernel(Geom g, const float4* __restrict__ U, FieldPtr A,
                                                             FieldPtr b, FieldPtr x, FieldPtr r_out, double* partial,
                                                             long long ps, const int* __restrict__ mask) {
  __shared__ double sh[32];
  if (mask && !mask[blockIdx.y]) return;
  const long long o = (long long)blockIdx.y * g.V * 12;  // double2 / float4 elements per field
  const double2* bb = (const double2*)b.data + o;
  const float4* xx = (const float4*)x.data + o;
  double2* rr = (double2*)r_out.data + o;
  partial += blockIdx.y * ps;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double nrm = 0;
  if (s < g.V) {
    const int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
    SpinAcc acc;
    df_site<0>(g, U, A, xx, blk, r, df_site_info(g, blk, r), acc);
    const long long e = (long long)blk * 12 * g.Vb + r;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const double2 bv = __ldg(bb + e + (long long)q * g.Vb);
      const double2 v = make_double2(bv.x - df_to_f64(acc_df(acc.re[q / 3][q % 3])),
                                     bv.y - df_to_f64(acc_df(acc.im[q / 3][q % 3])));
      rr[e + (long long)q * g.Vb] = v;
      nrm = fma(v.x, v.x, fma(v.y, v.y, nrm));
    }
  }
  const double t = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// r = b - D x (FP64), partial[blockIdx.x] = sum |r|^2 over the CTA; blockIdx.y
// selects a right-hand side of a batch (fields V sites apart, partial sums ps
// doubles apart), skipped when masked out
__global__ void __launch_bounds__(256) residual64_kernel(Geom g, const void* __restrict__ U, FieldPtr A, FieldPtr b,
                                                         FieldPtr x, FieldPtr r_out, double* partial, long long ps,
                                                         const int* __restrict__ mask) {
  __shared__ double sh[32];
  if (mask && !mask[blockIdx.y]) return;
  {
    const long long o = (long long)blockIdx.y * g.V * 12;  // double2 elements per FP64 field
    b.data = (double2*)b.data + o;
    x.data = (double2*)x.data + o;
    r_out.data = (double2*)r_out.data + o;
    partial += blockIdx.y * ps;
  }
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

int dirac_apply(qcd_ctx* c, const Rec& in, const Rec& out, int dagger, cudaStream_t s, int nrhs, const int* mask) {
  const int prec = in.prec;
  if (prec == PDF || (prec == P32 && out.prec == PDF)) {
    // the double-float operator: double-float in and out, or an FP32 input
    // (FP32-exact operand) with a double-float result
    if (out.prec != PDF || in.nreal != 24 || out.nreal != 24 || nrhs < 1) return QCD_ERR_ARG;
    QCD_TRY(ensure_gauge(c, PDF, s));
    QCD_TRY(ensure_clover(c, PDF, s));
    const bool in32 = prec == P32;
    const int threads = c->dirac_threads[PDF];
    const unsigned grid = (unsigned)((c->V + threads - 1) / threads);
    // algorithmic bytes: links and clover as pairs (576 + 576), spinor out 192, in 192 or 96
    ProfScope ps(c, QCD_KERNEL_DIRAC, s, (1344.0 + (in32 ? 96.0 : 192.0)) * (double)c->V * nrhs,
                 1824.0 * (double)c->V * nrhs);
    const float4* U = (const float4*)c->U[PDF];
    const FieldPtr A = c->A[PDF].ptr();
    if (in32) {
      if (dagger)
        dirac_df_kernel<1, true><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs, mask);
      else
        dirac_df_kernel<0, true><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs, mask);
    } else if (dagger) {
      dirac_df_kernel<1, false><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs, mask);
    } else {
      dirac_df_kernel<0, false><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs, mask);
    }
    QCD_LAUNCHED();
    return QCD_OK;
  }
  // FP64 in and double-float out: the FP64 operator with its result split
  const int out_df = prec == P64 && out.prec == PDF;
  if ((out.prec != prec && !out_df) || in.nreal != 24 || out.nreal != 24 || nrhs < 1) return QCD_ERR_ARG;
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
    dirac_kernel<PP, 1, BS><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs, mask, out_df); \
  else                                                                                                     \
    dirac_kernel<PP, 0, BS><<<grid, threads, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs, mask, out_df);
  // 16-bit storage (FP16, BF16) is issue-bound, so it gets the fixed-shape
  // instantiations, and the two-threads-per-site form when the context asks for it
  const int bs = block_shape_id(c->g);
  if ((prec == P16 || prec == PB16) && c->dirac_tps[prec] == 2) {
    const unsigned g2 = (unsigned)((c->V + kPairSites - 1) / kPairSites);
#define LAUNCH2(PP, DD, BB) \
  dirac_pair_kernel<PP, DD, BB><<<g2, 2 * kPairSites, 0, s>>>(c->g, U, A, in.ptr(), out.ptr(), nrhs, mask)
#define LAUNCH2_BS(PP, DD) \
  if (bs == 1) LAUNCH2(PP, DD, 1); else if (bs == 2) LAUNCH2(PP, DD, 2); else LAUNCH2(PP, DD, 0);
    if (prec == P16) {
      if (dagger) { LAUNCH2_BS(P16, 1) } else { LAUNCH2_BS(P16, 0) }
    } else {
      if (dagger) { LAUNCH2_BS(PB16, 1) } else { LAUNCH2_BS(PB16, 0) }
    }
#undef LAUNCH2_BS
#undef LAUNCH2
    QCD_LAUNCHED();
    return QCD_OK;
  }
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

int residual64(qcd_ctx* c, double* part, const Rec& b, const Rec& x, const Rec& r, double* d_norm2, cudaStream_t s,
               const Batch& B) {
  NvtxRange nv("residual64");
  if (b.prec != P64 || x.prec != P64 || r.prec != P64) return QCD_ERR_ARG;
  QCD_TRY(ensure_gauge(c, P64, s));
  QCD_TRY(ensure_clover(c, P64, s));
  const unsigned grid = (unsigned)((c->V + 255) / 256);
  {
    ProfScope ps(c, QCD_KERNEL_RESIDUAL, s, (bytes_per_site(P64) + 192) * (double)c->V * B.n,
                 1848.0 * (double)c->V * B.n);
    residual64_kernel<<<dim3(grid, B.n), 256, 0, s>>>(c->g, c->U[P64], c->A[P64].ptr(), b.ptr(), x.ptr(), r.ptr(),
                                                       part, B.ps, B.mask);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_norm2, s, B);
}

int residual_df(qcd_ctx* c, double* part, const Rec& b, const Rec& x, const Rec& r, const Rec& tmp, double* d_norm2,
                cudaStream_t s, const Batch& B, bool presplit) {
  NvtxRange nv("residual_df");
  if (b.prec != P64 || x.prec != P64 || r.prec != P64 || tmp.prec != PDF || tmp.bytes < (size_t)c->V * 192 * B.n)
    return QCD_ERR_ARG;
  QCD_TRY(ensure_gauge(c, PDF, s));
  QCD_TRY(ensure_clover(c, PDF, s));
  if (!presplit) QCD_TRY(blas_df_split(c, (const double*)x.data, (float*)tmp.data, s, B));
  const unsigned grid = (unsigned)((c->V + 255) / 256);
  {
    ProfScope ps(c, QCD_KERNEL_RESIDUAL, s, (bytes_per_site(P64) + 192) * (double)c->V * B.n,
                 1848.0 * (double)c->V * B.n);
    residual_df_kernel<<<dim3(grid, B.n), 256, 0, s>>>(c->g, (const float4*)c->U[PDF], c->A[PDF].ptr(), b.ptr(),
                                                        tmp.ptr(), r.ptr(), part, B.ps, B.mask);
    QCD_LAUNCHED();
  }
  return reduce_partials(part, (int)grid, 1, 1, d_norm2, s, B);
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
