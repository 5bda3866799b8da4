// Schwarz alternating procedure (Sec. 4) with even/odd MR block solves
// (Sec. 4: "the blocks are solved with a fixed number of iterations using a
// simple iterative solver (MR) and Dirichlet boundary conditions"; Sec. 5 /
// Table 1: even/odd preconditioning inside the block solver).
//
// One launch = one colour half-sweep: one CTA per block of that colour, one
// thread per (even site, odd site) pair.  The block's links and clover blocks
// are staged in shared memory, so the n_mr MR steps never touch HBM (Sec. 4:
// "all the data necessary for a block solve fit the local store").  With
// 16-bit block fields the staged copy keeps the storage format (two link rows,
// scaled clover halves) and is brought in by bulk (TMA) copies of the block's
// contiguous ranges; the third link row and the scales are applied on use.
// This halves the shared-memory footprint (two CTAs per SM) and the
// shared-memory bytes per hop.  FP32 and FP64 block fields are expanded to
// full matrices at stage-in.
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
  int* err;             // set to 1 if a staging wait timed out
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

// ------------------------------------------------------------------------
// Shared-memory copies of a block's links and clover blocks
// ------------------------------------------------------------------------

// FP32 / FP64: full matrices, SoA ([mu][18][Vb] links, [72][Vb] clover)
template <typename T>
struct ExpandedStage {
  T* U;
  T* A;
  int Vb;
  static constexpr size_t bytes(int Vb) { return sizeof(T) * (size_t)(4 * 18 + 72) * Vb; }
  __device__ __forceinline__ SU3<T> link(int r, int mu) const {
    SU3<T> u;
    const T* p = U + (mu * 18) * Vb + r;
#pragma unroll
    for (int k = 0; k < 9; ++k) u.m[k / 3][k % 3] = {p[(2 * k) * Vb], p[(2 * k + 1) * Vb]};
    return u;
  }
  __device__ __forceinline__ Spinor<T> clover(int r, const Spinor<T>& in) const {
    T c[72];
#pragma unroll
    for (int k = 0; k < 72; ++k) c[k] = A[k * Vb + r];
    return clover_apply(c, in);
  }
};

// 16-bit: the storage format itself -- links [4 mu][Vb] uint4 + [4 mu][Vb]
// uint2 (rows 0-1), clover [9][Vb] uint4 (scaled halves) + [Vb] float scales
template <int P>
struct HalfStage {
  const unsigned char* base;
  int Vb;
  typedef typename Storage<P>::real hr;
  static constexpr size_t bytes(int Vb) { return (size_t)(96 + 144 + 4) * Vb; }
  __device__ __forceinline__ SU3<float> link(int r, int mu) const {
    const uint4 a = ((const uint4*)base)[mu * Vb + r];
    const uint2 b = ((const uint2*)(base + 64 * Vb))[mu * Vb + r];
    const hr* ha = reinterpret_cast<const hr*>(&a);
    const hr* hb = reinterpret_cast<const hr*>(&b);
    SU3<float> u;
    u.m[0][0] = {to_f<P>(ha[0]), to_f<P>(ha[1])};
    u.m[0][1] = {to_f<P>(ha[2]), to_f<P>(ha[3])};
    u.m[0][2] = {to_f<P>(ha[4]), to_f<P>(ha[5])};
    u.m[1][0] = {to_f<P>(ha[6]), to_f<P>(ha[7])};
    u.m[1][1] = {to_f<P>(hb[0]), to_f<P>(hb[1])};
    u.m[1][2] = {to_f<P>(hb[2]), to_f<P>(hb[3])};
    reconstruct(u);
    return u;
  }
  __device__ __forceinline__ Spinor<float> clover(int r, const Spinor<float>& in) const {
    const uint4* A = (const uint4*)(base + 96 * Vb);
    float c[72];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const uint4 v = A[k * Vb + r];
      const hr* h = reinterpret_cast<const hr*>(&v);
#pragma unroll
      for (int e = 0; e < 8; ++e) c[8 * k + e] = to_f<P>(h[e]);
    }
    Spinor<float> o = clover_apply(c, in);
    const float s = ((const float*)(base + 240 * Vb))[r];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) o.c[a][b] = s * o.c[a][b];
    return o;
  }
};

// ------------------------------------------------------------------------
// bulk copy global -> shared with an mbarrier (TMA, non-tensor form)
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for phase 0 of the barrier for at most ~2^31 cycles (about a second)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, 0)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

// issue the bulk copies of a block's 16-bit links and clover (thread 0 only)
template <int P>
__device__ __forceinline__ void stage_issue(const SapArgs& a, int blk, unsigned char* dst, uint64_t* bar) {
  const int Vb = a.g.Vb;
  const unsigned char* srcs[3] = {(const unsigned char*)a.U + (size_t)blk * 96 * Vb,
                                  (const unsigned char*)a.Ahat.data + (size_t)blk * 144 * Vb,
                                  (const unsigned char*)(a.Ahat.norm + (size_t)blk * Vb)};
  const uint32_t sizes[3] = {(uint32_t)(96 * Vb), (uint32_t)(144 * Vb), (uint32_t)(4 * Vb)};
  mbar_expect_tx(bar, sizes[0] + sizes[1] + sizes[2]);
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    for (uint32_t o = 0; o < sizes[k]; o += 16384) {
      const uint32_t n = sizes[k] - o < 16384 ? sizes[k] - o : 16384;
      bulk_copy_g2s(dst + off + o, srcs[k] + o, n, bar);
    }
    off += sizes[k];
  }
}

// ------------------------------------------------------------------------
// block operator pieces
// ------------------------------------------------------------------------
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

// neighbour indices of one site packed two per int (16 bits each, 0xffff = outside)
__device__ __forceinline__ int nb_get(const int* pk, int k) {
  const int v = (pk[k >> 1] >> (16 * (k & 1))) & 0xffff;
  return v == 0xffff ? -1 : v;
}

// hops of D restricted to the block (Dirichlet: hops that leave the block are
// dropped) at site r from a field v on the opposite parity stored at
// src[index], index = neighbour site - off:
//   -1/2 sum_mu [U_mu(r)(1 - g) v(r + mu) + U_mu(r - mu)^+ (1 + g) v(r - mu)]
// One loop over mu (runtime spin phases): a single copy of the hop code.
template <typename T, typename ST>
__device__ __forceinline__ Spinor<T> hops(const ST& st, int n, int r, const T* src, const int* pk, int off) {
  Spinor<T> acc;
  zero(acc);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const SpinDir<T> d = spin_dir<T>(mu);
    const int kf = nb_get(pk, 2 * mu), kb = nb_get(pk, 2 * mu + 1);
    if (kf >= 0) {
      const Half<T> h = project_rt<-1>(s_spinor(src, n, kf), d);
      expand_add_rt<-1>(acc, umul(st.link(r, mu), h), T(1), d);
    }
    if (kb >= 0) {
      const Half<T> h = project_rt<+1>(s_spinor(src, n, kb), d);
      expand_add_rt<+1>(acc, udmul(st.link(kb + off, mu), h), T(1), d);
    }
  }
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
template <typename T, typename ST>
__device__ __forceinline__ void receive_faces(const SapArgs& a, const ST& st, int blk, int r, const int y[4],
                                              const int n[4], Spinor<T>& rho) {
  const Geom& g = a.g;
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const SpinDir<T> d = spin_dir<T>(mu);
    if (y[mu] == g.b[mu] - 1) {  // from block + mu: U_mu(y) (1 - g) part, projected by the sender
      const int nbk = n[mu] + 1 < g.nb[mu] ? blk + g.bstr[mu] : blk - (g.nb[mu] - 1) * g.bstr[mu];
      const Half<T> h = face_load<T>(a, nbk, 2 * mu, face_index(g, y, mu));
      expand_add_rt<-1>(rho, umul(st.link(r, mu), h), T(1), d);
    }
    if (y[mu] == 0) {  // from block - mu: U^+ (1 + g) part, multiplied by the sender
      const int nbk = n[mu] > 0 ? blk - g.bstr[mu] : blk + (g.nb[mu] - 1) * g.bstr[mu];
      const Half<T> w = face_load<T>(a, nbk, 2 * mu + 1, face_index(g, y, mu));
      expand_add_rt<+1>(rho, w, T(1), d);
    }
  }
}

// write the face contributions of the correction chi at site (blk, r)
template <typename T, typename ST>
__device__ __forceinline__ void send_faces(const SapArgs& a, const ST& st, int blk, int r, const int y[4],
                                           const int n[4], const Spinor<T>& chi) {
  const Geom& g = a.g;
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const SpinDir<T> d = spin_dir<T>(mu);
    if (y[mu] == 0) {  // to y = x - mu: 1/2 eta_mu(y) (1 - g) chi, projected
      const T f = T(0.5) * ((n[mu] == 0) ? (T)g.bc[mu] : T(1));
      Half<T> h = project_rt<-1>(chi, d);
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) h.c[s][c] = f * h.c[s][c];
      face_store<T>(a, blk, 2 * mu, face_index(g, y, mu), h);
    }
    if (y[mu] == g.b[mu] - 1) {  // to y = x + mu: 1/2 eta_mu(x) U_mu(x)^+ (1 + g) chi, projected
      const T f = T(0.5) * ((n[mu] == g.nb[mu] - 1) ? (T)g.bc[mu] : T(1));
      Half<T> w = udmul(st.link(r, mu), project_rt<+1>(chi, d));
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) w.c[s][c] = f * w.c[s][c];
      face_store<T>(a, blk, 2 * mu + 1, face_index(g, y, mu), w);
    }
  }
}

template <int P>
struct StageFor {
  typedef HalfStage<P> type;
};
template <>
struct StageFor<P32> {
  typedef ExpandedStage<float> type;
};
template <>
struct StageFor<P64> {
  typedef ExpandedStage<double> type;
};

template <int P, typename T>
__global__ void __launch_bounds__(256) sap_sweep_kernel(SapArgs a) {
  typedef typename StageFor<P>::type ST;
  constexpr bool kHalf = (P == P16 || P == PB16);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Geom& g = a.g;
  const int Vb = g.Vb, Vbh = g.Vbh;

  // shared memory: staged block fields, then the FP vectors r (even), t (odd),
  // rho_o (odd source), the reduction scratch and the staging barrier
  ST st;
  const size_t stage_bytes = ST::bytes(Vb);
  if constexpr (kHalf) {
    st.base = smem_raw;
    st.Vb = Vb;
  } else {
    st.U = (T*)smem_raw;
    st.A = st.U + 4 * 18 * Vb;
    st.Vb = Vb;
  }
  T* s_r = (T*)(smem_raw + stage_bytes);
  T* s_t = s_r + 24 * Vbh;
  T* s_rho_o = s_t + 24 * Vbh;
  T* s_red = s_rho_o + 24 * Vbh;
  uint64_t* bar = (uint64_t*)(s_red + 3 * 32);

  // block of the requested colour: pairs (2k, 2k+1) differ in n3 only, hence in colour
  int blk = 2 * blockIdx.x;
  int n[4];
  block_coords(g, blk, n);
  if (((n[0] + n[1] + n[2] + n[3]) & 1) != a.colour) {
    ++blk;
    ++n[3];
  }

  // ---- stage the block's links and clover
  if constexpr (kHalf) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      stage_issue<P>(a, blk, smem_raw, bar);
    }
  } else {
    for (int r = threadIdx.x; r < Vb; r += blockDim.x) {
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {
        SU3<T> u = load_link<P, T>(a.U, Vb, blk, r, mu);
        T* p = st.U + (mu * 18) * Vb + r;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          p[(2 * k) * Vb] = u.m[k / 3][k % 3].re;
          p[(2 * k + 1) * Vb] = u.m[k / 3][k % 3].im;
        }
      }
      T c[72];
      load_record<P, 72, T>(a.Ahat, Vb, blk, r, c);
#pragma unroll
      for (int k = 0; k < 72; ++k) st.A[k * Vb + r] = c[k];
    }
  }

  // thread i owns even site i and odd site Vbh + i; threads i >= Vbh (only
  // when a block has fewer than 64 sites) take part in barriers and sums only
  const int i = threadIdx.x;
  const bool act = i < Vbh;
  const int re = act ? i : 0, ro = act ? Vbh + i : Vbh;

  // ---- in-block neighbour tables of the two owned sites (while the copies fly)
  int ye[4], yo[4];
  {
    const int pe = __ldg(g.r2y + re), po = __ldg(g.r2y + ro);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      ye[mu] = ycoord(pe, mu);
      yo[mu] = ycoord(po, mu);
    }
  }
  // even site: indices into the odd vector t (site - Vbh); odd site: into r (= site)
  int pke[4], pko[4];
  {
    const int je = ye[0] * g.ystr[0] + ye[1] * g.ystr[1] + ye[2] * g.ystr[2] + ye[3] * g.ystr[3];
    const int jo = yo[0] * g.ystr[0] + yo[1] * g.ystr[1] + yo[2] * g.ystr[2] + yo[3] * g.ystr[3];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int ef = ye[mu] + 1 < g.b[mu] ? __ldg(g.j2r + je + g.ystr[mu]) - Vbh : 0xffff;
      const int eb = ye[mu] > 0 ? __ldg(g.j2r + je - g.ystr[mu]) - Vbh : 0xffff;
      const int of = yo[mu] + 1 < g.b[mu] ? __ldg(g.j2r + jo + g.ystr[mu]) : 0xffff;
      const int ob = yo[mu] > 0 ? __ldg(g.j2r + jo - g.ystr[mu]) : 0xffff;
      pke[mu] = ef | (eb << 16);
      pko[mu] = of | (ob << 16);
    }
  }

  // ---- residual of the two sites
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
  }
  if constexpr (kHalf) {
    // every thread waits (bounded) for the staging copies; a time-out is made
    // block-uniform, recorded, and the block is skipped
    const bool ok = mbar_wait_bounded(bar);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      mbar_wait_bounded(bar);  // let copies still in flight land before the CTA exits
      return;
    }
  } else {
    __syncthreads();
  }
  if (act) {
    if (a.faces_in) {
      receive_faces<T>(a, st, blk, re, ye, n, rho_e);
      receive_faces<T>(a, st, blk, ro, yo, n, rho_o);
    }
    s_spinor_store(s_rho_o, Vbh, i, rho_o);
    // etahat = rho_e - D_eo A_oo^-1 rho_o: first t = A_oo^-1 rho_o
    s_spinor_store(s_t, Vbh, i, st.clover(ro, rho_o));
  }
  __syncthreads();
  Spinor<T> r, x;
  zero(r);
  zero(x);
  if (act) {
    const Spinor<T> q = hops<T>(st, Vbh, re, s_t, pke, Vbh);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) r.c[s][c] = rho_e.c[s][c] - q.c[s][c];
    s_spinor_store(s_r, Vbh, i, r);
  }
  __syncthreads();

  // ---- MR on Dhat = A_ee - D_eo A_oo^-1 D_oe, x_e = 0, r = etahat.  Each
  // step runs two phases through one code path: phase 0 (odd sites)
  // t = A_oo^-1 D_oe r, phase 1 (even sites) p = A_ee r - D_eo t.
#pragma unroll 1
  for (int step = 0; step < 2 * a.nmr; ++step) {
    const int ph = step & 1;
    Spinor<T> p;
    zero(p);
    if (act) {
      const Spinor<T> hq = ph ? hops<T>(st, Vbh, re, s_t, pke, Vbh) : hops<T>(st, Vbh, ro, s_r, pko, 0);
      const Spinor<T> cl = st.clover(ph ? re : ro, ph ? r : hq);
      if (ph == 0) {
        s_spinor_store(s_t, Vbh, i, cl);
      } else {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) p.c[s][c] = cl.c[s][c] - hq.c[s][c];
      }
    }
    if (ph == 0) {
      __syncthreads();
      continue;
    }
    T pr_re = 0, pr_im = 0, pp = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cpx<T> v = p.c[s][c], w = r.c[s][c];
        pr_re += v.re * w.re + v.im * w.im;
        pr_im += v.re * w.im - v.im * w.re;
        pp += v.re * v.re + v.im * v.im;
      }
    cta_sum3(pr_re, pr_im, pp, s_red);
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
      s_spinor_store(s_r, Vbh, i, r);
    }
    __syncthreads();
  }

  // ---- chi_o = A_oo^-1 (rho_o - D_oe chi_e)
  if (act) s_spinor_store(s_r, Vbh, i, x);
  __syncthreads();
  if (!act) return;
  Spinor<T> chi_o;
  {
    Spinor<T> u = hops<T>(st, Vbh, ro, s_r, pko, 0);
    const Spinor<T> src = s_spinor(s_rho_o, Vbh, i);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) u.c[s][c] = src.c[s][c] - u.c[s][c];
    chi_o = st.clover(ro, u);
  }

  // ---- outputs: solution, block residual (r on even, 0 on odd), faces
  constexpr int PS = PsiPrec<P>::value;
  typedef typename std::conditional<PS == P64, double, float>::type TS;
#pragma unroll 1
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
      Spinor<double> dv;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) dv.c[s][c] = {(double)v.c[s][c].re, (double)v.c[s][c].im};
      store_spinor<P64, double>(a.out, Vb, blk, rs, dv);
    }
  }
  if (a.write_rho) {
    store_spinor<P, T>(a.rho, Vb, blk, re, r);
    Spinor<T> z;
    zero(z);
    store_spinor<P, T>(a.rho, Vb, blk, ro, z);
  }
  if (a.faces_out) {
    send_faces<T>(a, st, blk, re, ye, n, x);
    send_faces<T>(a, st, blk, ro, yo, n, chi_o);
  }
}

template <int P, typename T>
static size_t sap_smem_bytes(const Geom& g) {
  typedef typename StageFor<P>::type ST;
  return ST::bytes(g.Vb) + sizeof(T) * (3 * 24 * (size_t)g.Vbh + 3 * 32) + 16;
}

template <int P, typename T>
static int launch_sweep(const SapArgs& a, unsigned grid, int threads, cudaStream_t s, int maxsm) {
  const size_t smem = sap_smem_bytes<P, T>(a.g);
  if (smem > (size_t)maxsm) return QCD_ERR_UNSUPPORTED;
  QCD_CUDA(cudaFuncSetAttribute(sap_sweep_kernel<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sap_sweep_kernel<P, T><<<grid, threads, smem, s>>>(a);
  return QCD_OK;
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
  int dev = 0, maxsm = 0;
  QCD_CUDA(cudaGetDevice(&dev));
  QCD_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
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
  a.err = (int*)(c->d_scalars + 128);
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
  // flops (the 1320 + 504 convention): per solved site the Schur operator
  // costs about one D per MR step, plus about one more D for the source and
  // the back-substitution
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
      int st;
      switch (prec) {
        case P64: st = launch_sweep<P64, double>(a, grid, threads, s, maxsm); break;
        case P32: st = launch_sweep<P32, float>(a, grid, threads, s, maxsm); break;
        case P16: st = launch_sweep<P16, float>(a, grid, threads, s, maxsm); break;
        case PB16: st = launch_sweep<PB16, float>(a, grid, threads, s, maxsm); break;
        default: return QCD_ERR_ARG;
      }
      if (st != QCD_OK) return st;
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
