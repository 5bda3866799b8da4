// Device-side building blocks shared by the qcdgb kernels: complex arithmetic,
// lattice geometry, the block-major even/odd field layout, chiral-basis spin
// projection and precision-specific field access.
//
// Layout (Sec. 5: "points belonging to the same block are contiguous; inside
// the blocks, lattice points are divided into two sets, even and odd"):
//   internal site s = blk * Vb + r, blk = lexicographic Schwarz-block index
//   (block coordinate n3 fastest), r < Vb/2 even sites, r >= Vb/2 odd sites,
//   each parity ordered by the in-block lexicographic index j >> 1.
//   A field with NC 16-byte chunks per site is stored [blk][chunk][r]: one
//   block's data is one contiguous range (a single bulk copy stages it) and
//   consecutive threads touch consecutive 16-byte words (coalesced).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qcd {

enum Prec : int { P64 = 0, P32 = 1, P16 = 2, PB16 = 3, PDF = 4 };  // PDF: double-float pairs, FP64 layout

// ------------------------------------------------------------------------
// FP64 <-> FP32 conversion on the integer pipes.  GB300 runs FP64 conversions
// on its FP64 unit (2 per clock per SM), which turns kernels that convert a
// few dozen values per thread into FP64-bound ones; these do the IEEE-754
// conversion with integer operations for every normal result and hand the
// rare rest (zero handled here; subnormal results, infinities, NaN) to the
// hardware conversion, so the results are identical to it.
// ------------------------------------------------------------------------
// double -> float, round to nearest even: the 52-bit fraction is cut to 23
// bits; the dropped 29 bits decide the rounding, and a carry out of the
// fraction increments the exponent (reaching infinity past the largest float)
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e = (hi >> 20) & 0x7ffu;  // biased FP64 exponent
  if (e - 897u <= 253u) {                   // FP32 biased exponent e - 896 in 1 .. 254
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu, half = 0x10000000u;
    uint32_t r = ((e - 896u) << 23) | m;
    r += (uint32_t)(rem > half) | ((uint32_t)(rem == half) & (m & 1u));
    return __uint_as_float((hi & 0x80000000u) | r);
  }
  if ((b << 1) == 0ull) return __uint_as_float(hi & 0x80000000u);  // +-0
  return __double2float_rn(x);
}

// float -> double (exact): rebias the exponent, widen the fraction
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e - 1u <= 253u)  // normal
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
  if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);  // +-0
  return (double)f;
}

// ------------------------------------------------------------------------
// Double-float ("df64") numbers: x = hi + lo with two FP32 values, |lo| at
// most half an ulp of hi, a 48-bit significand carried on the FP32 pipes.
// Built from the error-free transformations: Knuth's TwoSum (s + e = a + b
// exactly), its Dekker form for |a| >= |b|, and the product split by a fused
// multiply-add (p + e = a b exactly, e = fma(a, b, -p)).  Used for the Krylov
// recursion of the solver, whose FP64 form is bound by GB300's FP64 rate.
// ------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| (or a = 0)
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
// x + y, with the two error terms folded into one renormalisation
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
// FP64 -> df64 (hi = x rounded to FP32, lo = the rest rounded) and back, on
// the integer pipes except one FP64 subtraction
__device__ __forceinline__ df df_from_f64(double x) {
  const float h = f64_to_f32(x);
  return {h, f64_to_f32(x - f32_to_f64(h))};
}
__device__ __forceinline__ double df_to_f64(df x) { return f32_to_f64(x.hi) + f32_to_f64(x.lo); }
// x y (the lo x lo term, 2^-48 relative, is dropped)
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
// z + x y
__device__ __forceinline__ df df_fma(df x, df y, df z) {
  df p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  df s = two_sum(z.hi, p.hi);
  s.lo += z.lo + p.lo;
  return fast_two_sum(s.hi, s.lo);
}

// A double-float running sum for long dot products: the high parts of the
// terms are added by TwoSum, every lower-order term (a product's rounding
// error, the cross terms, the sums' errors) is collected in c.  Neither part
// is renormalised until the value is read.
struct dfacc {
  float s, c;
};
// a += x y for double-floats x = (xh, xl), y = (yh, yl) (xl yl dropped)
__device__ __forceinline__ void acc_prod(dfacc& a, float xh, float xl, float yh, float yl) {
  const df p = two_prod(xh, yh);
  const df t = two_sum(a.s, p.hi);
  a.s = t.hi;
  a.c += t.lo + fmaf(xh, yl, fmaf(xl, yh, p.lo));
}
// a += (hi, lo)
__device__ __forceinline__ void acc_add(dfacc& a, float hi, float lo) {
  const df t = two_sum(a.s, hi);
  a.s = t.hi;
  a.c += t.lo + lo;
}
__device__ __forceinline__ double acc_value(const dfacc& a) { return f32_to_f64(a.s) + f32_to_f64(a.c); }
__device__ __forceinline__ df acc_df(const dfacc& a) { return two_sum(a.s, a.c); }

// ------------------------------------------------------------------------
// complex arithmetic
// ------------------------------------------------------------------------
template <typename T>
struct cpx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) { return cpx<T>{r, i}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a) { return {-a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
// a * b
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// c + a * b
template <typename T>
__device__ __forceinline__ cpx<T> cmadd(cpx<T> a, cpx<T> b, cpx<T> c) {
  return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
// c + conj(a) * b
template <typename T>
__device__ __forceinline__ cpx<T> cjmadd(cpx<T> a, cpx<T> b, cpx<T> c) {
  return {fma(a.re, b.re, fma(a.im, b.im, c.re)), fma(a.re, b.im, fma(-a.im, b.re, c.im))};
}
template <typename T>
__device__ __forceinline__ cpx<T> conjg(cpx<T> a) { return {a.re, -a.im}; }
// i * a
template <typename T>
__device__ __forceinline__ cpx<T> ti(cpx<T> a) { return {-a.im, a.re}; }
// -i * a
template <typename T>
__device__ __forceinline__ cpx<T> mti(cpx<T> a) { return {a.im, -a.re}; }

template <typename T>
struct Spinor {
  cpx<T> c[4][3];  // [spin][colour]
};
template <typename T>
struct Half {
  cpx<T> c[2][3];  // two spin components after projection
};
template <typename T>
struct SU3 {
  cpx<T> m[3][3];
};

template <typename T>
__device__ __forceinline__ void zero(Spinor<T>& s) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) s.c[a][b] = {T(0), T(0)};
}

// third row of an SU(3) matrix from the first two: row2 = conj(row0 x row1)
template <typename T>
__device__ __forceinline__ void reconstruct(SU3<T>& u) {
  u.m[2][0] = conjg(cmul(u.m[0][1], u.m[1][2]) - cmul(u.m[0][2], u.m[1][1]));
  u.m[2][1] = conjg(cmul(u.m[0][2], u.m[1][0]) - cmul(u.m[0][0], u.m[1][2]));
  u.m[2][2] = conjg(cmul(u.m[0][0], u.m[1][1]) - cmul(u.m[0][1], u.m[1][0]));
}

// w = U h  (two spin components)
template <typename T>
__device__ __forceinline__ Half<T> umul(const SU3<T>& u, const Half<T>& h) {
  Half<T> w;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<T> v = cmul(u.m[a][0], h.c[s][0]);
      v = cmadd(u.m[a][1], h.c[s][1], v);
      v = cmadd(u.m[a][2], h.c[s][2], v);
      w.c[s][a] = v;
    }
  return w;
}

// w = U^+ h
template <typename T>
__device__ __forceinline__ Half<T> udmul(const SU3<T>& u, const Half<T>& h) {
  Half<T> w;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<T> v = {T(0), T(0)};
      v = cjmadd(u.m[0][a], h.c[s][0], v);
      v = cjmadd(u.m[1][a], h.c[s][1], v);
      v = cjmadd(u.m[2][a], h.c[s][2], v);
      w.c[s][a] = v;
    }
  return w;
}

// FP32 overloads on packed FP32x2 arithmetic (sm_100 family): the two spin
// components of h travel in the two lanes, so each multiply-add by a link
// entry (broadcast to both lanes) serves both components.
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

__device__ __forceinline__ Half<float> umul(const SU3<float>& u, const Half<float>& h) {
  float2 hr[3], hi[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    hr[b] = make_float2(h.c[0][b].re, h.c[1][b].re);
    hi[b] = make_float2(h.c[0][b].im, h.c[1][b].im);
  }
  Half<float> w;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 wr = __fmul2_rn(bc2(u.m[a][0].re), hr[0]);
    float2 wi = __fmul2_rn(bc2(u.m[a][0].re), hi[0]);
    wr = __ffma2_rn(bc2(-u.m[a][0].im), hi[0], wr);
    wi = __ffma2_rn(bc2(u.m[a][0].im), hr[0], wi);
#pragma unroll
    for (int b = 1; b < 3; ++b) {
      wr = __ffma2_rn(bc2(u.m[a][b].re), hr[b], __ffma2_rn(bc2(-u.m[a][b].im), hi[b], wr));
      wi = __ffma2_rn(bc2(u.m[a][b].re), hi[b], __ffma2_rn(bc2(u.m[a][b].im), hr[b], wi));
    }
    w.c[0][a] = {wr.x, wi.x};
    w.c[1][a] = {wr.y, wi.y};
  }
  return w;
}

__device__ __forceinline__ Half<float> udmul(const SU3<float>& u, const Half<float>& h) {
  float2 hr[3], hi[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    hr[b] = make_float2(h.c[0][b].re, h.c[1][b].re);
    hi[b] = make_float2(h.c[0][b].im, h.c[1][b].im);
  }
  Half<float> w;
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // w_a = sum_b conj(u_ba) h_b
    float2 wr = __fmul2_rn(bc2(u.m[0][a].re), hr[0]);
    float2 wi = __fmul2_rn(bc2(u.m[0][a].re), hi[0]);
    wr = __ffma2_rn(bc2(u.m[0][a].im), hi[0], wr);
    wi = __ffma2_rn(bc2(-u.m[0][a].im), hr[0], wi);
#pragma unroll
    for (int b = 1; b < 3; ++b) {
      wr = __ffma2_rn(bc2(u.m[b][a].re), hr[b], __ffma2_rn(bc2(u.m[b][a].im), hi[b], wr));
      wi = __ffma2_rn(bc2(u.m[b][a].re), hi[b], __ffma2_rn(bc2(-u.m[b][a].im), hr[b], wi));
    }
    w.c[0][a] = {wr.x, wi.x};
    w.c[1][a] = {wr.y, wi.y};
  }
  return w;
}

// ------------------------------------------------------------------------
// Spin projection in the chiral basis.  Every g_mu has the form
// [[0, B], [B^+, 0]] with B unitary (B = -1, -i s1, -i s2, -i s3 for
// mu = 0..3), so (1 + S g_mu) psi = [h ; S B^+ h] with h = psi_u + S B psi_l:
// the projected spinor is carried by its two upper spin components.
// ------------------------------------------------------------------------
template <int MU, int S, typename T>
__device__ __forceinline__ Half<T> project(const Spinor<T>& p) {
  Half<T> h;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (MU == 0) {  // B psi_l = (-psi2, -psi3)
      h.c[0][a] = (S > 0) ? p.c[0][a] - p.c[2][a] : p.c[0][a] + p.c[2][a];
      h.c[1][a] = (S > 0) ? p.c[1][a] - p.c[3][a] : p.c[1][a] + p.c[3][a];
    } else if (MU == 1) {  // B psi_l = (-i psi3, -i psi2)
      h.c[0][a] = (S > 0) ? p.c[0][a] + mti(p.c[3][a]) : p.c[0][a] + ti(p.c[3][a]);
      h.c[1][a] = (S > 0) ? p.c[1][a] + mti(p.c[2][a]) : p.c[1][a] + ti(p.c[2][a]);
    } else if (MU == 2) {  // B psi_l = (-psi3, psi2)
      h.c[0][a] = (S > 0) ? p.c[0][a] - p.c[3][a] : p.c[0][a] + p.c[3][a];
      h.c[1][a] = (S > 0) ? p.c[1][a] + p.c[2][a] : p.c[1][a] - p.c[2][a];
    } else {  // B psi_l = (-i psi2, i psi3)
      h.c[0][a] = (S > 0) ? p.c[0][a] + mti(p.c[2][a]) : p.c[0][a] + ti(p.c[2][a]);
      h.c[1][a] = (S > 0) ? p.c[1][a] + ti(p.c[3][a]) : p.c[1][a] + mti(p.c[3][a]);
    }
  }
  return h;
}

// acc += f z and acc += f (i z) for real f: two fused multiply-adds per complex
template <typename T>
__device__ __forceinline__ void fadd(cpx<T>& acc, T f, const cpx<T>& z) {
  acc = {fma(f, z.re, acc.re), fma(f, z.im, acc.im)};
}
template <typename T>
__device__ __forceinline__ void fadd_i(cpx<T>& acc, T f, const cpx<T>& z) {
  acc = {fma(-f, z.im, acc.re), fma(f, z.re, acc.im)};
}

// acc += coef * [w ; S B^+ w]   (inverse of project<MU, S>); B^+ w is
// (-w0, -w1), (i w1, i w0), (w1, -w0), (i w0, -i w1) for mu = 0..3, and the
// coefficient and sign go into fused multiply-adds
template <int MU, int S, typename T>
__device__ __forceinline__ void expand_add(Spinor<T>& acc, const Half<T>& w, T coef) {
  const T f = S > 0 ? coef : -coef;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cpx<T> w0 = w.c[0][a], w1 = w.c[1][a];
    fadd(acc.c[0][a], coef, w0);
    fadd(acc.c[1][a], coef, w1);
    if (MU == 0) {
      fadd(acc.c[2][a], -f, w0);
      fadd(acc.c[3][a], -f, w1);
    } else if (MU == 1) {
      fadd_i(acc.c[2][a], f, w1);
      fadd_i(acc.c[3][a], f, w0);
    } else if (MU == 2) {
      fadd(acc.c[2][a], f, w1);
      fadd(acc.c[3][a], -f, w0);
    } else {
      fadd_i(acc.c[2][a], f, w0);
      fadd_i(acc.c[3][a], -f, w1);
    }
  }
}

// ------------------------------------------------------------------------
// Geometry
// ------------------------------------------------------------------------
struct Geom {
  int L[4];         // lattice extents, L[0] = time
  int b[4];         // Schwarz block extents (even)
  int nb[4];        // blocks per direction (even)
  int bstr[4];      // stride of block coordinate mu in the block index
  int ystr[4];      // stride of local coordinate mu in the in-block lexicographic index
  int Vb, Vbh;      // sites per block, half of it
  int nblk;         // number of blocks
  long long V;      // lattice volume
  double bc[4];     // sign of the hop that wraps around direction mu
  float bcf[4];     // the same signs in FP32 (no FP64 conversion in FP32 kernels)
  const int* r2y;   // r -> packed local coordinates (8 bits each, mu = 0 lowest)
  const int* j2r;   // in-block lexicographic index -> r
};

__device__ __forceinline__ int ycoord(int packed, int mu) { return (packed >> (8 * mu)) & 0xff; }

__device__ __forceinline__ void block_coords(const Geom& g, int blk, int n[4]) {
  int t = blk;
  n[3] = t % g.nb[3]; t /= g.nb[3];
  n[2] = t % g.nb[2]; t /= g.nb[2];
  n[1] = t % g.nb[1];
  n[0] = t / g.nb[1];
}

// boundary sign of direction mu in the arithmetic type
template <typename T>
__device__ __forceinline__ T bc_of(const Geom& g, int mu);
template <>
__device__ __forceinline__ double bc_of<double>(const Geom& g, int mu) { return g.bc[mu]; }
template <>
__device__ __forceinline__ float bc_of<float>(const Geom& g, int mu) { return g.bcf[mu]; }

struct Nbr {
  int blk, r;
  bool wrap;  // the hop crosses the lattice boundary in its direction
};

// neighbour of site (blk, r) with local coordinates y and block coordinates n,
// one step in direction mu (dir = +1 forward, -1 backward)
__device__ __forceinline__ Nbr neighbour(const Geom& g, int blk, const int y[4], const int n[4], int mu, int dir) {
  int j = y[0] * g.ystr[0] + y[1] * g.ystr[1] + y[2] * g.ystr[2] + y[3] * g.ystr[3];
  Nbr o;
  o.wrap = false;
  o.blk = blk;
  if (dir > 0) {
    if (y[mu] + 1 < g.b[mu]) {
      j += g.ystr[mu];
    } else {
      j -= (g.b[mu] - 1) * g.ystr[mu];
      if (n[mu] + 1 < g.nb[mu]) {
        o.blk += g.bstr[mu];
      } else {
        o.blk -= (g.nb[mu] - 1) * g.bstr[mu];
        o.wrap = true;
      }
    }
  } else {
    if (y[mu] > 0) {
      j -= g.ystr[mu];
    } else {
      j += (g.b[mu] - 1) * g.ystr[mu];
      if (n[mu] > 0) {
        o.blk -= g.bstr[mu];
      } else {
        o.blk += (g.nb[mu] - 1) * g.bstr[mu];
        o.wrap = true;
      }
    }
  }
  // even block extents: in-block lexicographic sites 2m and 2m + 1 differ only in
  // y3, hence in parity, so a site's rank among its parity is j >> 1; the
  // neighbour has the opposite parity (same rule as the j2r table, no load)
  const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  o.r = (par ^ 1) * g.Vbh + (j >> 1);
  return o;
}

// internal index of the site with global coordinates x (0 <= x_mu < L_mu)
__device__ __forceinline__ long long internal_index(const Geom& g, const int x[4]) {
  int blk = 0, j = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    blk += (x[mu] / g.b[mu]) * g.bstr[mu];
    j += (x[mu] % g.b[mu]) * g.ystr[mu];
  }
  return (long long)blk * g.Vb + __ldg(g.j2r + j);
}

__device__ __forceinline__ void global_coords(const Geom& g, int blk, int r, int x[4]) {
  int n[4];
  block_coords(g, blk, n);
  int p = __ldg(g.r2y + r);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) x[mu] = n[mu] * g.b[mu] + ycoord(p, mu);
}

__device__ __forceinline__ long long lex_index(const Geom& g, const int x[4]) {
  return ((long long)(x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

// ------------------------------------------------------------------------
// Field access.  A field is a base pointer plus (for 16-bit storage) a
// per-site FP32 scale array.  Element e of a record of N reals lives in
// chunk e / (16 / sizeof(storage)) of the site.
// ------------------------------------------------------------------------
struct FieldPtr {
  void* data;
  float* norm;  // per-site scale (16-bit storage only), indexed by internal site
};

template <int P>
struct Storage;
template <>
struct Storage<P64> {
  typedef double real;
  static constexpr int per_chunk = 2;
};
template <>
struct Storage<P32> {
  typedef float real;
  static constexpr int per_chunk = 4;
};
template <>
struct Storage<PDF> {  // two double-float reals (hi, lo, hi, lo) per 16-byte chunk
  typedef float real;
  static constexpr int per_chunk = 2;
};
template <>
struct Storage<P16> {
  typedef __half real;
  static constexpr int per_chunk = 8;
};
template <>
struct Storage<PB16> {
  typedef __nv_bfloat16 real;
  static constexpr int per_chunk = 8;
};

template <int P>
__device__ __forceinline__ float to_f(typename Storage<P>::real v);
template <>
__device__ __forceinline__ float to_f<P16>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f<PB16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <int P>
__device__ __forceinline__ typename Storage<P>::real from_f(float v);
template <>
__device__ __forceinline__ __half from_f<P16>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<PB16>(float v) { return __float2bfloat16_rn(v); }

// a packed pair of 16-bit reals -> two FP32 values
template <int P>
__device__ __forceinline__ float2 to_f2(uint32_t w);
template <>
__device__ __forceinline__ float2 to_f2<P16>(uint32_t w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
}
template <>
__device__ __forceinline__ float2 to_f2<PB16>(uint32_t w) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
}

// load N reals (N a multiple of the chunk width) of site (blk, r) of a field
// with NC chunks per site; T is the arithmetic type
template <int P, int N, typename T>
__device__ __forceinline__ void load_record(const FieldPtr& f, int Vb, int blk, int r, T* out) {
  constexpr int W = Storage<P>::per_chunk;
  constexpr int NC = (N + W - 1) / W;
  const long long base = (long long)blk * NC * Vb + r;
  if constexpr (P == P64) {
    const double2* d = (const double2*)f.data;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      double2 v = __ldg(d + base + (long long)k * Vb);
      out[2 * k] = (T)v.x;
      out[2 * k + 1] = (T)v.y;
    }
  } else if constexpr (P == PDF) {
    const float4* d = (const float4*)f.data;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const float4 v = __ldg(d + base + (long long)k * Vb);
      out[2 * k] = (T)df_to_f64(df{v.x, v.y});
      out[2 * k + 1] = (T)df_to_f64(df{v.z, v.w});
    }
  } else if constexpr (P == P32) {
    const float4* d = (const float4*)f.data;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      float4 v = __ldg(d + base + (long long)k * Vb);
      out[4 * k] = v.x;
      out[4 * k + 1] = v.y;
      out[4 * k + 2] = v.z;
      out[4 * k + 3] = v.w;
    }
  } else {
    const uint4* d = (const uint4*)f.data;
    const float s = f.norm ? __ldg(f.norm + (long long)blk * Vb + r) : 1.0f;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      uint4 v = __ldg(d + base + (long long)k * Vb);
      const typename Storage<P>::real* h = reinterpret_cast<const typename Storage<P>::real*>(&v);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (8 * k + e < N) out[8 * k + e] = s * to_f<P>(h[e]);
    }
  }
}

// N reals of a 16-bit record without its per-site scale applied; returns the
// scale (1 when the field has none), so callers can fold it into a later
// multiplication
template <int P, int N>
__device__ __forceinline__ float load_record_raw(const FieldPtr& f, int Vb, int blk, int r, float* out) {
  static_assert(P == P16 || P == PB16, "16-bit storage only");
  constexpr int NC = (N + 7) / 8;
  const long long base = (long long)blk * NC * Vb + r;
  const uint4* d = (const uint4*)f.data;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const uint4 v = __ldg(d + base + (long long)k * Vb);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (8 * k + 2 * e < N) {
        const float2 x = to_f2<P>(w[e]);
        out[8 * k + 2 * e] = x.x;
        out[8 * k + 2 * e + 1] = x.y;
      }
  }
  return f.norm ? __ldg(f.norm + (long long)blk * Vb + r) : 1.0f;
}

// store N reals; 16-bit storage computes the per-site max-abs scale
template <int P, int N, typename T>
__device__ __forceinline__ void store_record(const FieldPtr& f, int Vb, int blk, int r, const T* in) {
  constexpr int W = Storage<P>::per_chunk;
  constexpr int NC = (N + W - 1) / W;
  const long long base = (long long)blk * NC * Vb + r;
  if constexpr (P == P64) {
    double2* d = (double2*)f.data;
#pragma unroll
    for (int k = 0; k < NC; ++k) d[base + (long long)k * Vb] = make_double2((double)in[2 * k], (double)in[2 * k + 1]);
  } else if constexpr (P == PDF) {
    float4* d = (float4*)f.data;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const df a = df_from_f64((double)in[2 * k]), b = df_from_f64((double)in[2 * k + 1]);
      d[base + (long long)k * Vb] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
  } else if constexpr (P == P32) {
    float4* d = (float4*)f.data;
#pragma unroll
    for (int k = 0; k < NC; ++k)
      d[base + (long long)k * Vb] = make_float4((float)in[4 * k], (float)in[4 * k + 1], (float)in[4 * k + 2], (float)in[4 * k + 3]);
  } else {
    float m = 0.f;
#pragma unroll
    for (int e = 0; e < N; ++e) m = fmaxf(m, fabsf((float)in[e]));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* d = (uint4*)f.data;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      uint4 v;
      typename Storage<P>::real* h = reinterpret_cast<typename Storage<P>::real*>(&v);
#pragma unroll
      for (int e = 0; e < 8; ++e) h[e] = from_f<P>(8 * k + e < N ? (float)in[8 * k + e] * inv : 0.f);
      d[base + (long long)k * Vb] = v;
    }
    f.norm[(long long)blk * Vb + r] = m;
  }
}

// spinor: 24 reals, component (spin s, colour c) at reals 6 s + 2 c
template <int P, typename T>
__device__ __forceinline__ Spinor<T> load_spinor(const FieldPtr& f, int Vb, int blk, int r) {
  T v[24];
  load_record<P, 24, T>(f, Vb, blk, r, v);
  Spinor<T> s;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) s.c[a][b] = {v[6 * a + 2 * b], v[6 * a + 2 * b + 1]};
  return s;
}

template <int P, typename T>
__device__ __forceinline__ void store_spinor(const FieldPtr& f, int Vb, int blk, int r, const Spinor<T>& s) {
  T v[24];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      v[6 * a + 2 * b] = s.c[a][b].re;
      v[6 * a + 2 * b + 1] = s.c[a][b].im;
    }
  store_record<P, 24, T>(f, Vb, blk, r, v);
}

// ------------------------------------------------------------------------
// Gauge field.  FP64: full 18 reals per link ([blk][mu][9 double2][r]), since
// the FP64 operator is bound by FP64 arithmetic, not bytes.  FP32: rows 0-1
// (12 reals, [blk][mu][3 float4][r]).  16-bit: rows 0-1 as 8 + 4 values,
// [blk][mu][r] uint4 followed by [blk][mu][r] uint2, no scale (|U_ab| <= 1).
// ------------------------------------------------------------------------
template <int P>
struct GaugeLayout;
template <>
struct GaugeLayout<P64> {
  static constexpr long long bytes_per_site = 4 * 18 * 8;
};
template <>
struct GaugeLayout<P32> {
  static constexpr long long bytes_per_site = 4 * 12 * 4;
};
template <>
struct GaugeLayout<P16> {
  static constexpr long long bytes_per_site = 4 * 12 * 2;
};
template <>
struct GaugeLayout<PB16> {
  static constexpr long long bytes_per_site = 4 * 12 * 2;
};

template <int P, typename T>
__device__ __forceinline__ SU3<T> load_link(const void* U, int Vb, int blk, int r, int mu) {
  SU3<T> u;
  if constexpr (P == P64) {
    const double2* d = (const double2*)U + ((long long)(blk * 4 + mu) * 9) * Vb + r;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = __ldg(d + (long long)k * Vb);
      u.m[k / 3][k % 3] = {(T)v.x, (T)v.y};
    }
  } else if constexpr (P == P32) {
    const float4* d = (const float4*)U + ((long long)(blk * 4 + mu) * 3) * Vb + r;
    float f[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 v = __ldg(d + (long long)k * Vb);
      f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) u.m[k / 3][k % 3] = {(T)f[2 * k], (T)f[2 * k + 1]};
    reconstruct(u);
  } else {
    typedef typename Storage<P>::real hr;
    const char* base = (const char*)U + (long long)blk * Vb * 96;
    uint4 a = __ldg((const uint4*)base + (long long)mu * Vb + r);
    uint2 b = __ldg((const uint2*)(base + (long long)64 * Vb) + (long long)mu * Vb + r);
    const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float2 x = to_f2<P>(w[k]);
      u.m[k / 3][k % 3] = {(T)x.x, (T)x.y};
    }
    reconstruct(u);
  }
  return u;
}

// ------------------------------------------------------------------------
// Clover: two Hermitian 6x6 chiral blocks, 36 reals each: 6 diagonal reals,
// then the 15 upper off-diagonal elements (i < j, row-major) as (re, im).
// Block 0 acts on spins 0-1, block 1 on spins 2-3; index within a block is
// (spin % 2) * 3 + colour.
// ------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void clover_block_apply(const T* c, const cpx<T>* in, cpx<T>* out) {
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] = c[i] * in[i];
  int k = 6;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      cpx<T> a = {c[k], c[k + 1]};
      k += 2;
      out[i] = cmadd(a, in[j], out[i]);
      out[j] = cjmadd(a, in[i], out[j]);
    }
}

template <typename T>
__device__ __forceinline__ Spinor<T> clover_apply(const T* c72, const Spinor<T>& p) {
  Spinor<T> o;
  cpx<T> in[6], out[6];
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
#pragma unroll
    for (int i = 0; i < 6; ++i) in[i] = p.c[2 * blk + i / 3][i % 3];
    clover_block_apply(c72 + 36 * blk, in, out);
#pragma unroll
    for (int i = 0; i < 6; ++i) o.c[2 * blk + i / 3][i % 3] = out[i];
  }
  return o;
}

}  // namespace qcd

namespace qcd {

// ------------------------------------------------------------------------
// Runtime-direction form of the projection above, for kernels that loop over
// mu instead of instantiating four copies (smaller code).  In the chiral
// basis B psi_l has components ph_k psi_{sigma_k}: (sigma_0, sigma_1) = (2, 3)
// or (3, 2) ("swap") and phases ph_k in {+-1, +-i}; the expansion puts
// conj(ph_k) w_k on spin sigma_k.
// ------------------------------------------------------------------------
template <typename T>
struct SpinDir {
  bool swap;
  cpx<T> ph0, ph1;
};

template <typename T>
__device__ __forceinline__ SpinDir<T> spin_dir(int mu) {
  SpinDir<T> d;
  const T o = T(1), z = T(0);
  switch (mu) {
    case 0: d.swap = false; d.ph0 = {-o, z}; d.ph1 = {-o, z}; break;  // B = -1
    case 1: d.swap = true; d.ph0 = {z, -o}; d.ph1 = {z, -o}; break;   // B = -i s1
    case 2: d.swap = true; d.ph0 = {-o, z}; d.ph1 = {o, z}; break;    // B = -i s2
    default: d.swap = false; d.ph0 = {z, -o}; d.ph1 = {z, o}; break;  // B = -i s3
  }
  return d;
}

// h = upper components of (1 + S g_mu) p
template <int S, typename T>
__device__ __forceinline__ Half<T> project_rt(const Spinor<T>& p, const SpinDir<T>& d) {
  Half<T> h;
  const cpx<T> a0 = {T(S) * d.ph0.re, T(S) * d.ph0.im}, a1 = {T(S) * d.ph1.re, T(S) * d.ph1.im};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cpx<T> l0 = d.swap ? p.c[3][c] : p.c[2][c];
    const cpx<T> l1 = d.swap ? p.c[2][c] : p.c[3][c];
    h.c[0][c] = cmadd(a0, l0, p.c[0][c]);
    h.c[1][c] = cmadd(a1, l1, p.c[1][c]);
  }
  return h;
}

// acc += coef * [w ; S B^+ w]
template <int S, typename T>
__device__ __forceinline__ void expand_add_rt(Spinor<T>& acc, const Half<T>& w, T coef, const SpinDir<T>& d) {
  const cpx<T> b0 = {T(S) * coef * d.ph0.re, -T(S) * coef * d.ph0.im};
  const cpx<T> b1 = {T(S) * coef * d.ph1.re, -T(S) * coef * d.ph1.im};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc.c[0][c] = acc.c[0][c] + coef * w.c[0][c];
    acc.c[1][c] = acc.c[1][c] + coef * w.c[1][c];
    const cpx<T> l0 = cmul(b0, w.c[0][c]), l1 = cmul(b1, w.c[1][c]);
    acc.c[2][c] = acc.c[2][c] + (d.swap ? l1 : l0);
    acc.c[3][c] = acc.c[3][c] + (d.swap ? l0 : l1);
  }
}

}  // namespace qcd
