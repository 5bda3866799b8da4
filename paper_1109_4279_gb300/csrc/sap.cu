// Schwarz alternating procedure (Sec. 4) with even/odd MR block solves
// (Sec. 4: "the blocks are solved with a fixed number of iterations using a
// simple iterative solver (MR) and Dirichlet boundary conditions"; Sec. 5 /
// Table 1: even/odd preconditioning inside the block solver).
//
// One launch = one colour half-sweep: one CTA per block of that colour, one
// thread per (even site, odd site) pair.  The block's links, clover blocks and
// residual are staged in shared memory, so the n_mr MR steps never touch HBM
// (Sec. 4: "all the data necessary for a block solve fit the local store").
//
// Residual update on the neighbouring blocks (Sec. 4: "the residue is then
// updated ... on the internal border of the black blocks") goes through face
// buffers, the one-GPU analogue of the paper's per-block-border receive
// buffers (Sec. 5): each solved block writes, for every site on each of its 8
// faces, the spin-projected (6 complex) hop of its correction into its own
// face buffer; blocks of the other colour add them to their residual when
// they are staged in the next half-sweep.  Corner sites receive from several
// blocks without races, and the sum order is fixed (deterministic).
#include <type_traits>

#include "internal.h"

namespace qcd {

struct SapArgs {
  Geom g;
  int colour;           // blocks with (n0 + n1 + n2 + n3) % 2 == colour are solved
  int nmr;              // MR steps per block
  int read_eta;         // residual source: 1 = eta (FP64), 0 = rho_sap
  int faces_in;         // add face contributions of the other colour
  int faces_out;        // write this block's face contributions
  int write_rho;        // store the block residual
  int psi_mode;         // 0: psi_sap = chi; 1: psi_sap += chi; 2: out64 = chi; 3: out64 = psi_sap + chi
  const void* U;        // links in the SAP storage precision
  FieldPtr Ahat;        // A on even sites, A^-1 on odd sites
  FieldPtr eta;         // FP64 source
  FieldPtr rho;         // residual, SAP storage precision
  FieldPtr psi;         // accumulated solution (FP32, or FP64 for the FP64 variant)
  FieldPtr out;         // FP64 result
  void* faces;          // [blk][NCF chunks][F] face data
  int F;                // face sites per block
  int fo[8];            // offset of face 2 mu + dir inside a block's face list
};

template <typename T>
struct FaceChunks {
  static constexpr int n = 12 * (int)sizeof(T) / 16;  // chunks of 16 bytes per face site
};

// face site index: lexicographic over the local coordinates other than mu
__device__ __forceinline__ int face_index(const Geom& g, const int y[4], int mu) {
  int q = 0;
#pragma unroll
  for (int nu = 0; nu < 4; ++nu)
    if (nu != mu) q = q * g.b[nu] + y[nu];
  return q;
}

template <typename T>
__device__ __forceinline__ void face_store(const SapArgs& a, int blk, int f, int q, const Half<T>& h) {
  T v[12];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[6 * s + 2 * c] = h.c[s][c].re;
      v[6 * s + 2 * c + 1] = h.c[s][c].im;
    }
  const long long base = (long long)blk * FaceChunks<T>::n * a.F + a.fo[f] + q;
  if constexpr (sizeof(T) == 8) {
    double2* d = (double2*)a.faces;
#pragma unroll
    for (int k = 0; k < 6; ++k) d[base + (long long)k * a.F] = make_double2(v[2 * k], v[2 * k + 1]);
  } else {
    float4* d = (float4*)a.faces;
#pragma unroll
    for (int k = 0; k < 3; ++k) d[base + (long long)k * a.F] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  }
}

template <typename T>
__device__ __forceinline__ Half<T> face_load(const SapArgs& a, int blk, int f, int q) {
  T v[12];
  const long long base = (long long)blk * FaceChunks<T>::n * a.F + a.fo[f] + q;
  if constexpr (sizeof(T) == 8) {
    const double2* d = (const double2*)a.faces;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double2 t = d[base + (long long)k * a.F];
      v[2 * k] = t.x;
      v[2 * k + 1] = t.y;
    }
  } else {
    const float4* d = (const float4*)a.faces;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 t = d[base + (long long)k * a.F];
      v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    }
  }
  Half<T> h;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) h.c[s][c] = {v[6 * s + 2 * c], v[6 * s + 2 * c + 1]};
  return h;
}

// shared-memory block fields, SoA so that consecutive threads hit consecutive banks
template <typename T>
struct Smem {
  T* U;     // [4 mu][18][Vb]
  T* A;     // [72][Vb]
  T* r;     // [24][Vbh] even-site MR residual
  T* t;     // [24][Vbh] odd-site temporary
  T* rho_o; // [24][Vbh] odd-site source
  T* red;   // reduction scratch
};

template <typename T>
__device__ __forceinline__ SU3<T> s_link(const Smem<T>& sm, int Vb, int r, int mu) {
  SU3<T> u;
  const T* p = sm.U + (long long)mu * 18 * Vb + r;
#pragma unroll
  for (int k = 0; k < 9; ++k) u.m[k / 3][k % 3] = {p[(2 * k) * Vb], p[(2 * k + 1) * Vb]};
  return u;
}

template <typename T>
__device__ __forceinline__ Spinor<T> s_spinor(const T* base, int n, int i) {
  Spinor<T> s;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) s.c[a][b] = {base[(6 * a + 2 * b) * n + i], base[(6 * a + 2 * b + 1) * n + i]};
  return s;
}

template <typename T>
__device__ __forceinline__ void s_spinor_store(T* base, int n, int i, const Spinor<T>& s) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      base[(6 * a + 2 * b) * n + i] = s.c[a][b].re;
      base[(6 * a + 2 * b + 1) * n + i] = s.c[a][b].im;
    }
}

template <typename T>
__device__ __forceinline__ Spinor<T> s_clover(const Smem<T>& sm, int Vb, int r, const Spinor<T>& p) {
  T c[72];
#pragma unroll
  for (int k = 0; k < 72; ++k) c[k] = sm.A[k * Vb + r];
  return clover_apply(c, p);
}

// hops of D restricted to the block (Dirichlet: hops that leave the block are
// dropped) evaluated at site r from a field living on the opposite parity:
// returns -1/2 sum_mu [U_mu(r)(1 - g) v(r + mu) + U_mu(r - mu)^+ (1 + g) v(r - mu)]
// nb[2 mu + 0/1]: forward/backward neighbour's index into `src` (-1 if outside),
// nr[2 mu + 1]: backward neighbour's site index r (for its link)
template <int MU, typename T>
__device__ __forceinline__ void block_hop(const Smem<T>& sm, int Vb, int n, int r, const T* src, const int* nb,
                                          const int* nr, Spinor<T>& acc) {
  if (nb[2 * MU] >= 0) {
    Spinor<T> p = s_spinor(src, n, nb[2 * MU]);
    Half<T> h = project<MU, -1>(p);
    Half<T> w = umul(s_link(sm, Vb, r, MU), h);
    expand_add<MU, -1>(acc, w, T(1));
  }
  if (nb[2 * MU + 1] >= 0) {
    Spinor<T> p = s_spinor(src, n, nb[2 * MU + 1]);
    Half<T> h = project<MU, +1>(p);
    Half<T> w = udmul(s_link(sm, Vb, nr[2 * MU + 1], MU), h);
    expand_add<MU, +1>(acc, w, T(1));
  }
}

template <typename T>
__device__ __forceinline__ Spinor<T> hops(const Smem<T>& sm, int Vb, int n, int r, const T* src, const int* nb,
                                          const int* nr) {
  Spinor<T> acc;
  zero(acc);
  block_hop<0, T>(sm, Vb, n, r, src, nb, nr, acc);
  block_hop<1, T>(sm, Vb, n, r, src, nb, nr, acc);
  block_hop<2, T>(sm, Vb, n, r, src, nb, nr, acc);
  block_hop<3, T>(sm, Vb, n, r, src, nb, nr, acc);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.c[s][c] = T(-0.5) * acc.c[s][c];
  return acc;
}

// deterministic CTA-wide sum of 3 values; every thread gets the totals
template <typename T>
__device__ __forceinline__ void cta_sum3(T& a, T& b, T& c, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[3 * w] = a;
    red[3 * w + 1] = b;
    red[3 * w + 2] = c;
  }
  __syncthreads();
  a = b = c = T(0);
  for (int k = 0; k < nw; ++k) {
    a += red[3 * k];
    b += red[3 * k + 1];
    c += red[3 * k + 2];
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void add_spinor(Spinor<T>& a, const Spinor<T>& b, T s) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) a.c[i][c] = a.c[i][c] + s * b.c[i][c];
}

// psi storage precision of the SAP accumulator
template <int P>
struct PsiPrec {
  static constexpr int value = P32;
};
template <>
struct PsiPrec<P64> {
  static constexpr int value = P64;
};

// receive the face contributions of the other colour at site (blk, r)
template <typename T>
__device__ __forceinline__ void receive_faces(const SapArgs& a, const Smem<T>& sm, int blk, int r, const int y[4],
                                              const int n[4], Spinor<T>& rho) {
  const Geom& g = a.g;
#define RECV(MU)                                                                             \
  if (y[MU] == g.b[MU] - 1) {                                                                \
    int nbk = n[MU] + 1 < g.nb[MU] ? blk + g.bstr[MU] : blk - (g.nb[MU] - 1) * g.bstr[MU];   \
    Half<T> h = face_load<T>(a, nbk, 2 * MU, face_index(g, y, MU));                          \
    expand_add<MU, -1>(rho, umul(s_link(sm, g.Vb, r, MU), h), T(1));                         \
  }                                                                                          \
  if (y[MU] == 0) {                                                                          \
    int nbk = n[MU] > 0 ? blk - g.bstr[MU] : blk + (g.nb[MU] - 1) * g.bstr[MU];              \
    Half<T> w = face_load<T>(a, nbk, 2 * MU + 1, face_index(g, y, MU));                      \
    expand_add<MU, +1>(rho, w, T(1));                                                        \
  }
  RECV(0) RECV(1) RECV(2) RECV(3)
#undef RECV
}

// write the face contributions of the correction chi at site (blk, r)
template <typename T>
__device__ __forceinline__ void send_faces(const SapArgs& a, const Smem<T>& sm, int blk, int r, const int y[4],
                                           const int n[4], const Spinor<T>& chi) {
  const Geom& g = a.g;
#define SEND(MU)                                                                                  \
  if (y[MU] == 0) { /* to y = x - mu: 1/2 eta_mu(y) (1 - g) chi, projected */                     \
    const T eta = (n[MU] == 0) ? (T)g.bc[MU] : T(1);                                              \
    Half<T> h = project<MU, -1>(chi);                                                             \
    _Pragma("unroll") for (int s = 0; s < 2; ++s)                                                 \
      _Pragma("unroll") for (int c = 0; c < 3; ++c) h.c[s][c] = (T(0.5) * eta) * h.c[s][c];       \
    face_store<T>(a, blk, 2 * MU, face_index(g, y, MU), h);                                       \
  }                                                                                               \
  if (y[MU] == g.b[MU] - 1) { /* to y = x + mu: 1/2 eta_mu(x) U_mu(x)^+ (1 + g) chi, projected */ \
    const T eta = (n[MU] == g.nb[MU] - 1) ? (T)g.bc[MU] : T(1);                                   \
    Half<T> w = udmul(s_link(sm, g.Vb, r, MU), project<MU, +1>(chi));                             \
    _Pragma("unroll") for (int s = 0; s < 2; ++s)                                                 \
      _Pragma("unroll") for (int c = 0; c < 3; ++c) w.c[s][c] = (T(0.5) * eta) * w.c[s][c];       \
    face_store<T>(a, blk, 2 * MU + 1, face_index(g, y, MU), w);                                   \
  }
  SEND(0) SEND(1) SEND(2) SEND(3)
#undef SEND
}

template <int P, typename T>
__global__ void __launch_bounds__(256) sap_sweep_kernel(SapArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geom& g = a.g;
  const int Vb = g.Vb, Vbh = g.Vbh;
  Smem<T> sm;
  sm.U = (T*)smem_raw;
  sm.A = sm.U + 4 * 18 * Vb;
  sm.r = sm.A + 72 * Vb;
  sm.t = sm.r + 24 * Vbh;
  sm.rho_o = sm.t + 24 * Vbh;
  sm.red = sm.rho_o + 24 * Vbh;

  // block of the requested colour: pairs (2k, 2k+1) differ in n3 only, hence in colour
  int blk = 2 * blockIdx.x;
  int n[4];
  block_coords(g, blk, n);
  if (((n[0] + n[1] + n[2] + n[3]) & 1) != a.colour) {
    ++blk;
    ++n[3];
  }
  // thread i owns even site i and odd site Vbh + i; threads i >= Vbh (only
  // when a block has fewer than 64 sites) take part in barriers and sums only
  const int i = threadIdx.x;
  const bool act = i < Vbh;
  const int re = act ? i : 0, ro = act ? Vbh + i : Vbh;

  // ---- stage links and clover of the block in shared memory
  for (int r = i; r < Vb; r += blockDim.x) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      SU3<T> u = load_link<P, T>(a.U, Vb, blk, r, mu);
      T* p = sm.U + (long long)mu * 18 * Vb + r;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        p[(2 * k) * Vb] = u.m[k / 3][k % 3].re;
        p[(2 * k + 1) * Vb] = u.m[k / 3][k % 3].im;
      }
    }
    T c[72];
    load_record<P, 72, T>(a.Ahat, Vb, blk, r, c);
#pragma unroll
    for (int k = 0; k < 72; ++k) sm.A[k * Vb + r] = c[k];
  }

  // ---- in-block neighbour tables of the two owned sites
  int ye[4], yo[4];
  {
    const int pe = __ldg(g.r2y + re), po = __ldg(g.r2y + ro);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      ye[mu] = ycoord(pe, mu);
      yo[mu] = ycoord(po, mu);
    }
  }
  // even site: nbe = index into the odd vector t, nre = site index (links);
  // odd site: nbo = index into the even vector r (= site index)
  int nbe[8], nre[8], nbo[8];
  {
    const int je = ye[0] * g.ystr[0] + ye[1] * g.ystr[1] + ye[2] * g.ystr[2] + ye[3] * g.ystr[3];
    const int jo = yo[0] * g.ystr[0] + yo[1] * g.ystr[1] + yo[2] * g.ystr[2] + yo[3] * g.ystr[3];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      int f = ye[mu] + 1 < g.b[mu] ? __ldg(g.j2r + je + g.ystr[mu]) : -1;
      int b = ye[mu] > 0 ? __ldg(g.j2r + je - g.ystr[mu]) : -1;
      nbe[2 * mu] = f >= 0 ? f - Vbh : -1;
      nbe[2 * mu + 1] = b >= 0 ? b - Vbh : -1;
      nre[2 * mu] = f;
      nre[2 * mu + 1] = b;
      nbo[2 * mu] = yo[mu] + 1 < g.b[mu] ? __ldg(g.j2r + jo + g.ystr[mu]) : -1;
      nbo[2 * mu + 1] = yo[mu] > 0 ? __ldg(g.j2r + jo - g.ystr[mu]) : -1;
    }
  }
  __syncthreads();

  // ---- residual of the two sites (+ incoming faces)
  Spinor<T> rho_e, rho_o;
  zero(rho_e);
  zero(rho_o);
  if (act) {
    if (a.read_eta) {
      Spinor<double> d = load_spinor<P64, double>(a.eta, Vb, blk, re);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) rho_e.c[s][c] = {(T)d.c[s][c].re, (T)d.c[s][c].im};
      d = load_spinor<P64, double>(a.eta, Vb, blk, ro);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) rho_o.c[s][c] = {(T)d.c[s][c].re, (T)d.c[s][c].im};
    } else {
      rho_e = load_spinor<P, T>(a.rho, Vb, blk, re);
      rho_o = load_spinor<P, T>(a.rho, Vb, blk, ro);
    }
    if (a.faces_in) {
      receive_faces<T>(a, sm, blk, re, ye, n, rho_e);
      receive_faces<T>(a, sm, blk, ro, yo, n, rho_o);
    }
    s_spinor_store(sm.rho_o, Vbh, i, rho_o);
    // etahat = rho_e - D_eo A_oo^-1 rho_o: first t = A_oo^-1 rho_o
    s_spinor_store(sm.t, Vbh, i, s_clover(sm, Vb, ro, rho_o));
  }
  __syncthreads();
  Spinor<T> r, x;
  zero(r);
  zero(x);
  if (act) {
    Spinor<T> q = hops(sm, Vb, Vbh, re, sm.t, nbe, nre);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) r.c[s][c] = rho_e.c[s][c] - q.c[s][c];
    s_spinor_store(sm.r, Vbh, i, r);
  }
  __syncthreads();

  // ---- MR on Dhat = A_ee - D_eo A_oo^-1 D_oe, x_e = 0, r = etahat
  for (int it = 0; it < a.nmr; ++it) {
    // odd site: t = A_oo^-1 D_oe r
    if (act) {
      Spinor<T> u = hops(sm, Vb, Vbh, ro, sm.r, nbo, nbo);
      s_spinor_store(sm.t, Vbh, i, s_clover(sm, Vb, ro, u));
    }
    __syncthreads();
    // even site: p = A_ee r - D_eo t; alpha = (p, r) / (p, p)
    T pr_re = 0, pr_im = 0, pp = 0;
    Spinor<T> p;
    zero(p);
    if (act) {
      p = s_clover(sm, Vb, re, r);
      Spinor<T> q = hops(sm, Vb, Vbh, re, sm.t, nbe, nre);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cpx<T> v = p.c[s][c] - q.c[s][c];
          p.c[s][c] = v;
          cpx<T> w = r.c[s][c];
          pr_re += v.re * w.re + v.im * w.im;
          pr_im += v.re * w.im - v.im * w.re;
          pp += v.re * v.re + v.im * v.im;
        }
    }
    cta_sum3(pr_re, pr_im, pp, sm.red);
    const T inv = pp > T(0) ? T(1) / pp : T(0);
    const cpx<T> alpha = {pr_re * inv, pr_im * inv};
    if (act) {
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          x.c[s][c] = cmadd(alpha, r.c[s][c], x.c[s][c]);
          r.c[s][c] = r.c[s][c] - cmul(alpha, p.c[s][c]);
        }
      s_spinor_store(sm.r, Vbh, i, r);
    }
    __syncthreads();
  }

  // ---- chi_o = A_oo^-1 (rho_o - D_oe chi_e)
  if (act) s_spinor_store(sm.r, Vbh, i, x);
  __syncthreads();
  if (!act) return;
  Spinor<T> chi_o;
  {
    Spinor<T> u = hops(sm, Vb, Vbh, ro, sm.r, nbo, nbo);
    Spinor<T> src = s_spinor(sm.rho_o, Vbh, i);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) u.c[s][c] = src.c[s][c] - u.c[s][c];
    chi_o = s_clover(sm, Vb, ro, u);
  }

  // ---- outputs: solution, block residual (r on even, 0 on odd), faces
  constexpr int PS = PsiPrec<P>::value;
  typedef typename std::conditional<PS == P64, double, float>::type TS;
  for (int half = 0; half < 2; ++half) {
    const int rs = half ? ro : re;
    const Spinor<T>& chi = half ? chi_o : x;
    Spinor<TS> v;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) v.c[s][c] = {(TS)chi.c[s][c].re, (TS)chi.c[s][c].im};
    if (a.psi_mode == 1 || a.psi_mode == 3) {
      Spinor<TS> old = load_spinor<PS, TS>(a.psi, Vb, blk, rs);
      add_spinor(v, old, TS(1));
    }
    if (a.psi_mode <= 1) {
      store_spinor<PS, TS>(a.psi, Vb, blk, rs, v);
    } else {
      Spinor<double> d;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) d.c[s][c] = {(double)v.c[s][c].re, (double)v.c[s][c].im};
      store_spinor<P64, double>(a.out, Vb, blk, rs, d);
    }
  }
  if (a.write_rho) {
    store_spinor<P, T>(a.rho, Vb, blk, re, r);
    Spinor<T> z;
    zero(z);
    store_spinor<P, T>(a.rho, Vb, blk, ro, z);
  }
  if (a.faces_out) {
    send_faces<T>(a, sm, blk, re, ye, n, x);
    send_faces<T>(a, sm, blk, ro, yo, n, chi_o);
  }
}

template <typename T>
static size_t sap_smem_bytes(const Geom& g) {
  return sizeof(T) * ((size_t)4 * 18 * g.Vb + 72 * (size_t)g.Vb + 3 * 24 * (size_t)g.Vbh + 3 * 32);
}

static int sap_apply_impl(qcd_ctx* c, SapWork& w, const Rec& eta64, const Rec& psi64, int ncy, int nmr, int prec,
                   cudaStream_t s) {
  const Geom& g = c->g;
  if (eta64.prec != P64 || psi64.prec != P64) return QCD_ERR_ARG;
  if (ncy < 1 || nmr < 0) return QCD_ERR_ARG;
  if (g.Vbh > 256) return QCD_ERR_UNSUPPORTED;
  QCD_TRY(ensure_gauge(c, prec, s));
  QCD_TRY(ensure_clover(c, prec, s));
  const bool dbl = prec == P64;
  const size_t smem = dbl ? sap_smem_bytes<double>(g) : sap_smem_bytes<float>(g);
  int dev = 0, maxsm = 0;
  QCD_CUDA(cudaGetDevice(&dev));
  QCD_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)maxsm) return QCD_ERR_UNSUPPORTED;
  // work fields
  if (w.prec != prec) {
    rec_free(w.rho);
    rec_free(w.psi);
    if (w.faces) cudaFree(w.faces);
    w.faces = nullptr;
    QCD_TRY(rec_alloc(w.rho, prec, 24, c->V));
    QCD_TRY(rec_alloc(w.psi, dbl ? P64 : P32, 24, c->V));
    int F = 0;
    for (int mu = 0; mu < 4; ++mu) F += 2 * (g.Vb / g.b[mu]);
    w.faces_bytes = (size_t)c->nblk * F * 12 * (dbl ? 8 : 4);
    if (cudaMalloc(&w.faces, w.faces_bytes) != cudaSuccess) {
      w.faces = nullptr;
      return QCD_ERR_NOMEM;
    }
    w.prec = prec;
  }
  SapArgs a;
  a.g = g;
  a.nmr = nmr;
  a.U = c->U[prec];
  a.Ahat = c->Ahat[prec].ptr();
  a.eta = eta64.ptr();
  a.rho = w.rho.ptr();
  a.psi = w.psi.ptr();
  a.out = psi64.ptr();
  a.faces = w.faces;
  int off = 0;
  for (int mu = 0; mu < 4; ++mu) {
    a.fo[2 * mu] = off;
    off += g.Vb / g.b[mu];
    a.fo[2 * mu + 1] = off;
    off += g.Vb / g.b[mu];
  }
  a.F = off;
  const unsigned grid = (unsigned)(c->nblk / 2);
  const int threads = g.Vbh < 32 ? 32 : ((g.Vbh + 31) / 32) * 32;
  // flops: per site and MR step the Schur operator costs about one D (1824),
  // plus the source/back-substitution (about one more D) per sweep
  const double flops = (double)(nmr + 1) * 1824.0 * (double)c->V / 2.0;
  const double sb = dbl ? 8 : (prec == P32 ? 4 : 2);
  const double bytes = (double)c->V / 2 * (4 * (dbl ? 18 : 12) * sb + 72 * sb + 2 * 24 * sb + 2 * 24 * (dbl ? 8 : 4));
  for (int cy = 0; cy < ncy; ++cy)
    for (int colour = 0; colour < 2; ++colour) {
      const int h = 2 * cy + colour;
      a.colour = colour;
      a.read_eta = cy == 0;
      a.faces_in = h > 0;
      a.faces_out = h < 2 * ncy - 1;
      const bool last = cy == ncy - 1;
      a.write_rho = !last;
      a.psi_mode = last ? (cy == 0 ? 2 : 3) : (cy == 0 ? 0 : 1);
      ProfScope ps(c, QCD_KERNEL_SAP, s, bytes, flops);
      if (dbl) {
        QCD_CUDA(cudaFuncSetAttribute(sap_sweep_kernel<P64, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        sap_sweep_kernel<P64, double><<<grid, threads, smem, s>>>(a);
      } else {
        switch (prec) {
          case P32:
            QCD_CUDA(cudaFuncSetAttribute(sap_sweep_kernel<P32, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            sap_sweep_kernel<P32, float><<<grid, threads, smem, s>>>(a);
            break;
          case P16:
            QCD_CUDA(cudaFuncSetAttribute(sap_sweep_kernel<P16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            sap_sweep_kernel<P16, float><<<grid, threads, smem, s>>>(a);
            break;
          case PB16:
            QCD_CUDA(cudaFuncSetAttribute(sap_sweep_kernel<PB16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            sap_sweep_kernel<PB16, float><<<grid, threads, smem, s>>>(a);
            break;
          default: return QCD_ERR_ARG;
        }
      }
      QCD_LAUNCHED();
    }
  return QCD_OK;
}

int sap_apply(qcd_ctx* c, const Rec& eta64, const Rec& psi64, int ncy, int nmr, int prec, cudaStream_t s) {
  Workspace* ws = ensure_ws(c);
  if (!ws) return QCD_ERR_NOMEM;
  return sap_apply_impl(c, ws->sap, eta64, psi64, ncy, nmr, prec, s);
}

}  // namespace qcd
