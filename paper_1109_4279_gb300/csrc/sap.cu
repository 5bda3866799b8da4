// Schwarz alternating procedure (Sec. 4) with even/odd MR block solves
// (Sec. 4: "the blocks are solved with a fixed number of iterations using a
// simple iterative solver (MR) and Dirichlet boundary conditions"; Sec. 5 /
// Table 1: even/odd preconditioning inside the block solver).
//
// One launch = one colour half-sweep: one CTA per block of that colour, two
// threads per (even site, odd site) pair.  The block's links and clover blocks
// are staged in shared memory, so the n_mr MR steps never touch HBM (Sec. 4:
// "all the data necessary for a block solve fit the local store").  With
// 16-bit block fields the block's contiguous ranges arrive by bulk (TMA)
// copies: the two-row links are rebuilt once per block into full 16-bit
// matrices, the clover blocks stay in the storage format and their per-site
// scale is applied on use (112 KB per 4^4 block: two CTAs per SM; 224 KB per
// 8x4x4x4 block: one).  FP32 and FP64 block fields are expanded to full
// matrices at stage-in.
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
  int read_eta;         // residual source: 1 = eta, 0 = rho_sap
  int io32;             // eta and out are FP32 fields (else FP64)
  int io_df;            // eta and out are double-float fields (eta read as its FP32 high parts)
  int out32;            // with io_df: out is an FP32 field instead (the block solution is FP32-exact)
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
  long long wait_cycles;  // budget of the staging wait (clock cycles)
  int extra_tx;         // bytes the staging barrier expects beyond the copies (0; a test sets more)
  // right-hand sides: nrhs fields back to back in eta, rho, psi, out and the
  // face buffers (byte strides below; rho_ns: floats between 16-bit scale
  // arrays); CTA (x, y) solves block x for right-hand sides y rt .. y rt + rt - 1
  // in turn, with the block's links and clover staged once
  int nrhs, rt;
  const int* mask;      // device flags: right-hand side r is solved iff mask[r] != 0 (null: all)
  long long eta_rs, rho_rs, rho_ns, psi_rs, out_rs, faces_rs;
};

// the fields of right-hand side r (computed where used, so that no per-RHS
// pointer stays live across the block solve)
__device__ __forceinline__ FieldPtr rhs_eta(const SapArgs& a, int r) {
  return {(char*)a.eta.data + r * a.eta_rs, nullptr};
}
__device__ __forceinline__ FieldPtr rhs_rho(const SapArgs& a, int r) {
  return {(char*)a.rho.data + r * a.rho_rs, a.rho.norm ? a.rho.norm + r * a.rho_ns : nullptr};
}
__device__ __forceinline__ FieldPtr rhs_psi(const SapArgs& a, int r) {
  return {(char*)a.psi.data + r * a.psi_rs, nullptr};
}
__device__ __forceinline__ FieldPtr rhs_out(const SapArgs& a, int r) {
  return {(char*)a.out.data + r * a.out_rs, nullptr};
}
__device__ __forceinline__ void* rhs_faces(const SapArgs& a, int r) { return (char*)a.faces + r * a.faces_rs; }

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
__device__ __forceinline__ void face_store(const SapArgs& a, void* faces, int blk, int f, int q, const Half<T>& h) {
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
    double2* d = (double2*)faces;
#pragma unroll
    for (int k = 0; k < 6; ++k) d[base + (long long)k * a.F] = make_double2(v[2 * k], v[2 * k + 1]);
  } else {
    float4* d = (float4*)faces;
#pragma unroll
    for (int k = 0; k < 3; ++k) d[base + (long long)k * a.F] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  }
}

template <typename T>
__device__ __forceinline__ Half<T> face_load(const SapArgs& a, const void* faces, int blk, int f, int q) {
  T v[12];
  const long long base = (long long)blk * FaceChunks<T>::n * a.F + a.fo[f] + q;
  if constexpr (sizeof(T) == 8) {
    const double2* d = (const double2*)faces;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double2 t = d[base + (long long)k * a.F];
      v[2 * k] = t.x;
      v[2 * k + 1] = t.y;
    }
  } else {
    const float4* d = (const float4*)faces;
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
  __device__ __forceinline__ void base_init(unsigned char* p, int vb) {
    U = (T*)p;
    A = U + 4 * 18 * vb;
    Vb = vb;
  }
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

// 16-bit, links expanded once at stage-in: full matrices as 16-bit complex
// pairs, entries 0-7 in two 16-byte chunks [4 mu][2][Vb] and entry 8 in
// [4 mu][Vb] (three loads per link); the clover blocks in the storage format,
// [9][Vb] uint4 (scaled halves) + [Vb] float scales, applied on use.  The compressed
// links arrive by bulk copy in a landing zone and are rebuilt there into full
// matrices, so no hop pays for the third row.
template <int P>
struct HalfExpStage {
  const unsigned char* base;
  int Vb;
  __device__ __forceinline__ void base_init(unsigned char* p, int vb) {
    base = p;
    Vb = vb;
  }
  typedef typename Storage<P>::real hr;
  static constexpr size_t bytes(int Vb) { return (size_t)(144 + 144 + 4) * Vb; }
  __device__ __forceinline__ SU3<float> link(int r, int mu) const {
    const uint4* q = (const uint4*)base + (2 * mu) * Vb + r;
    const uint4 a = q[0], b = q[Vb];
    const uint32_t c = ((const uint32_t*)(base + 128 * Vb))[mu * Vb + r];
    const uint32_t w[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c};
    SU3<float> u;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float2 x = to_f2<P>(w[k]);
      u.m[k / 3][k % 3] = {x.x, x.y};
    }
    return u;
  }
  __device__ __forceinline__ const uint4* clover_chunks() const { return (const uint4*)(base + 144 * Vb); }
  __device__ __forceinline__ const float* clover_scales() const { return (const float*)(base + 288 * Vb); }
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

// wait for phase 0 of the barrier for at most `budget` clock cycles (2^31, about
// a second, unless a test asks for less)
static constexpr long long kWaitCycles = 1ll << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, 0)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// issue the bulk copies of a block's 16-bit links (to `links`) and clover
// blocks with their scales (to `clover`) on the barrier: every lane of warp 0
// calls this, lane 0 adds the expected bytes and lane c issues pieces c,
// c + 32, ... of at most 16 KB
template <int P>
__device__ __forceinline__ void stage_issue(const SapArgs& a, int blk, unsigned char* links, unsigned char* clover,
                                            uint64_t* bar) {
  const int Vb = a.g.Vb, lane = threadIdx.x & 31;
  const unsigned char* srcs[3] = {(const unsigned char*)a.U + (size_t)blk * 96 * Vb,
                                  (const unsigned char*)a.Ahat.data + (size_t)blk * 144 * Vb,
                                  (const unsigned char*)(a.Ahat.norm + (size_t)blk * Vb)};
  unsigned char* dsts[3] = {links, clover, clover + 144 * Vb};
  const uint32_t sizes[3] = {(uint32_t)(96 * Vb), (uint32_t)(144 * Vb), (uint32_t)(4 * Vb)};
  if (lane == 0) mbar_expect_tx(bar, sizes[0] + sizes[1] + sizes[2] + (uint32_t)a.extra_tx);
  __syncwarp();
  int c0 = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int nk = (int)((sizes[k] + 16383) / 16384);
    for (int c = (lane - c0 % 32 + 32) % 32; c < nk; c += 32) {
      const uint32_t o = (uint32_t)c * 16384, n = sizes[k] - o < 16384 ? sizes[k] - o : 16384;
      bulk_copy_g2s(dsts[k] + o, srcs[k] + o, n, bar);
    }
    c0 += nk;
  }
}

// L2 prefetch of a contiguous range (16-byte aligned start and size)
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// What a block reads only after its staging and block solve: the faces its
// eight neighbours wrote in the previous half-sweep and its accumulated
// solution.  With one CTA per SM nothing overlaps those loads, so the lanes of
// warp 1 ask for them in L2 at the start (one range per face, chunk and
// direction; the block's solution is one range), where the later loads find them.
template <typename T, int PS>
__device__ __forceinline__ void prefetch_late_reads(const SapArgs& a, const void* faces, const FieldPtr& psi, int blk,
                                                    const int n[4]) {
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31;
  constexpr int NCF = FaceChunks<T>::n;
  if (a.faces_in) {
    for (int t = lane; t < 8 * NCF; t += 32) {
      const int f = t / NCF, k = t - f * NCF, mu = f >> 1;
      const int nmu = mu == 0 ? n[0] : (mu == 1 ? n[1] : (mu == 2 ? n[2] : n[3]));  // no local-memory copy of n
      // face 2 mu comes from the block at +mu, face 2 mu + 1 from the block at -mu
      const int nbk = (f & 1) == 0 ? (nmu + 1 < g.nb[mu] ? blk + g.bstr[mu] : blk - (g.nb[mu] - 1) * g.bstr[mu])
                                   : (nmu > 0 ? blk - g.bstr[mu] : blk + (g.nb[mu] - 1) * g.bstr[mu]);
      const long long e = (long long)nbk * NCF * a.F + (long long)k * a.F + a.fo[f];
      prefetch_l2((const char*)faces + 16 * e, (uint32_t)(16 * (g.Vb / g.b[mu])));
    }
  }
  if ((a.psi_mode == 1 || a.psi_mode == 3) && lane == 31) {
    constexpr int NCH = PS == P64 ? 12 : 6;  // 16-byte chunks per site
    prefetch_l2((const char*)psi.data + (size_t)16 * NCH * g.Vb * blk, (uint32_t)(16 * NCH * g.Vb));
  }
}

// rebuild the compressed 16-bit links of the landing zone (rows 0-1, layout of
// the storage format) into full 16-bit matrices (HalfExpStage layout)
template <int P>
__device__ __forceinline__ void expand_links(const unsigned char* land, unsigned char* out, int Vb) {
  typedef typename Storage<P>::real hr;
  for (int r = threadIdx.x; r < Vb; r += blockDim.x) {
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      const uint4 a = ((const uint4*)land)[mu * Vb + r];
      const uint2 b = ((const uint2*)(land + 64 * Vb))[mu * Vb + r];
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
      uint32_t w[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        hr* h = reinterpret_cast<hr*>(&w[k]);
        h[0] = from_f<P>(u.m[k / 3][k % 3].re);
        h[1] = from_f<P>(u.m[k / 3][k % 3].im);
      }
      uint4* q = (uint4*)out + (2 * mu) * Vb + r;
      q[0] = make_uint4(w[0], w[1], w[2], w[3]);
      q[Vb] = make_uint4(w[4], w[5], w[6], w[7]);
      ((uint32_t*)(out + 128 * Vb))[mu * Vb + r] = w[8];
    }
  }
}

// ------------------------------------------------------------------------
// block operator pieces
// ------------------------------------------------------------------------
// Spinor fields in shared memory are stored as 16-byte chunks [24 / R][n]
// (R = 4 FP32 or 2 FP64 reals per chunk; real 6 a + 2 b (+1) is spin a,
// colour b), so a site's spinor is 6 (FP32) or 12 (FP64) vector loads.
template <typename T>
struct Chunk;
template <>
struct Chunk<float> {
  typedef float4 type;
  static constexpr int R = 4;
};
template <>
struct Chunk<double> {
  typedef double2 type;
  static constexpr int R = 2;
};

template <typename T>
__device__ __forceinline__ void chunk_get(const typename Chunk<T>::type& c, T* v);
template <>
__device__ __forceinline__ void chunk_get<float>(const float4& c, float* v) {
  v[0] = c.x;
  v[1] = c.y;
  v[2] = c.z;
  v[3] = c.w;
}
template <>
__device__ __forceinline__ void chunk_get<double>(const double2& c, double* v) {
  v[0] = c.x;
  v[1] = c.y;
}
__device__ __forceinline__ float4 chunk_make(const float* v) { return make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ double2 chunk_make(const double* v) { return make_double2(v[0], v[1]); }

// reals [k0, k0 + N) of site i of a chunked field with stride n
template <typename T, int N>
__device__ __forceinline__ void s_load(const T* base, int n, int i, int k0, T* v) {
  typedef typename Chunk<T>::type C;
  constexpr int R = Chunk<T>::R;
  const C* p = (const C*)base + (k0 / R) * n + i;
#pragma unroll
  for (int k = 0; k < N / R; ++k) chunk_get<T>(p[k * n], v + R * k);
}
template <typename T, int N>
__device__ __forceinline__ void s_store(T* base, int n, int i, int k0, const T* v) {
  typedef typename Chunk<T>::type C;
  constexpr int R = Chunk<T>::R;
  C* p = (C*)base + (k0 / R) * n + i;
#pragma unroll
  for (int k = 0; k < N / R; ++k) p[k * n] = chunk_make(v + R * k);
}

template <typename T>
__device__ __forceinline__ Spinor<T> s_spinor(const T* base, int n, int i) {
  T v[24];
  s_load<T, 24>(base, n, i, 0, v);
  Spinor<T> s;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) s.c[a][b] = {v[6 * a + 2 * b], v[6 * a + 2 * b + 1]};
  return s;
}

// ------------------------------------------------------------------------
// Pair split: the two threads of an (even site, odd site) pair share the work
// of every site operation.  Thread half hf computes the hops in directions
// mu = 2 hf and 2 hf + 1 (so no link is loaded twice) and owns spin
// components 2 hf and 2 hf + 1 of every vector; the clover term, being block
// diagonal in chirality, acts on the owned half alone.  The two threads of a
// pair sit in different warps (hf is warp-uniform, so the two direction sets
// never diverge inside a warp) and exchange their partial hop sums through
// shared memory.
// ------------------------------------------------------------------------

// owned half (spins 2 hf, 2 hf + 1: reals 12 hf .. 12 hf + 11) of a chunked
// spinor field in shared memory
template <typename T>
__device__ __forceinline__ Half<T> s_half(const T* base, int n, int i, int hf) {
  T v[12];
  s_load<T, 12>(base, n, i, 12 * hf, v);
  Half<T> h;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) h.c[s][c] = {v[6 * s + 2 * c], v[6 * s + 2 * c + 1]};
  return h;
}

template <typename T>
__device__ __forceinline__ void s_half_store(T* base, int n, int i, int hf, const Half<T>& h) {
  T v[12];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[6 * s + 2 * c] = h.c[s][c].re;
      v[6 * s + 2 * c + 1] = h.c[s][c].im;
    }
  s_store<T, 12>(base, n, i, 12 * hf, v);
}

template <typename T>
__device__ __forceinline__ Half<T> half_of(const Spinor<T>& v, int hf) {
  Half<T> h;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) h.c[s][c] = hf ? v.c[2 + s][c] : v.c[s][c];
  return h;
}

template <typename T>
__device__ __forceinline__ Half<T> half_axpy(const Half<T>& a, const Half<T>& b, T s) {  // a + s b
  Half<T> o;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) o.c[i][c] = a.c[i][c] + s * b.c[i][c];
  return o;
}

// clover chiral block hf applied to an owned half
template <typename T>
__device__ __forceinline__ Half<T> clover_half_apply(const T* c36, const Half<T>& in) {
  cpx<T> i6[6], o6[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) i6[k] = in.c[k / 3][k % 3];
  clover_block_apply(c36, i6, o6);
  Half<T> o;
#pragma unroll
  for (int k = 0; k < 6; ++k) o.c[k / 3][k % 3] = o6[k];
  return o;
}

template <typename T>
__device__ __forceinline__ Half<T> clover_half(const ExpandedStage<T>& st, int r, int hf, const Half<T>& in) {
  T c[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) c[k] = st.A[(36 * hf + k) * st.Vb + r];
  return clover_half_apply(c, in);
}

template <int P>
__device__ __forceinline__ Half<float> clover_half_native(const uint4* A, const float* scales, int Vb, int r, int hf,
                                                          const Half<float>& in) {
  // chunks 4 hf .. 4 hf + 4 hold this chiral block's 36 values (18 packed
  // pairs) starting at pair 2 hf
  uint32_t w20[20];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint4 v = A[(4 * hf + k) * Vb + r];
    w20[4 * k] = v.x;
    w20[4 * k + 1] = v.y;
    w20[4 * k + 2] = v.z;
    w20[4 * k + 3] = v.w;
  }
  float c[36];
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    const float2 f = to_f2<P>(hf ? w20[k + 2] : w20[k]);
    c[2 * k] = f.x;
    c[2 * k + 1] = f.y;
  }
  Half<float> o = clover_half_apply(c, in);
  const float s = scales[r];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) o.c[a][b] = s * o.c[a][b];
  return o;
}

template <int P>
__device__ __forceinline__ Half<float> clover_half(const HalfExpStage<P>& st, int r, int hf, const Half<float>& in) {
  return clover_half_native<P>(st.clover_chunks(), st.clover_scales(), st.Vb, r, hf, in);
}

// one direction of the block operator's hops at site r:
//   U_mu(r)(1 - g) v(r + mu) + U_mu(r - mu)^+ (1 + g) v(r - mu)
// (Dirichlet: hops leaving the block are absent); v lives on the opposite
// parity at src[site - off] (chunked, stride n); pm = forward | backward << 16
// indices into src.  A neighbour outside the block is the zero slot n - 1,
// so the hop adds nothing and the code has no data-dependent branch (its
// link is then the site's own, any valid link).
template <int MU, typename T, typename ST>
__device__ __forceinline__ void hop_dir(const ST& st, int n, int r, const T* src, int pm, int off, Spinor<T>& acc) {
  const int kf = pm & 0xffff, kb = (pm >> 16) & 0xffff;
  const int lb = kb == n - 1 ? r : kb + off;
  const Half<T> h0 = project<MU, -1>(s_spinor(src, n, kf));
  expand_add<MU, -1>(acc, umul(st.link(r, MU), h0), T(1));
  const Half<T> h1 = project<MU, +1>(s_spinor(src, n, kb));
  expand_add<MU, +1>(acc, udmul(st.link(lb, MU), h1), T(1));
}

// partial hops over this thread's directions 2 hf, 2 hf + 1 (hf is uniform
// across a warp, so both branches run without divergence)
template <typename T, typename ST>
__device__ __forceinline__ Spinor<T> hops_pair(const ST& st, int n, int r, const T* src, const int pk[2], int off,
                                               int hf) {
  Spinor<T> acc;
  zero(acc);
  if (hf) {
    hop_dir<2, T>(st, n, r, src, pk[0], off, acc);
    hop_dir<3, T>(st, n, r, src, pk[1], off, acc);
  } else {
    hop_dir<0, T>(st, n, r, src, pk[0], off, acc);
    hop_dir<1, T>(st, n, r, src, pk[1], off, acc);
  }
  return acc;
}

// Pair exchange through shared memory: xb holds [2][12][np] reals (np = site
// pairs per half, a multiple of 32).  Both calls below contain a barrier and
// must be reached by every thread of the CTA.

// barrier of the two warps that hold pairs 32 w .. 32 w + 31 (warp w of each
// half): named barrier 1 + w (np / 32 <= 8 of them; barrier 0 is the CTA-wide one)
__device__ __forceinline__ void pair_warps_sync(int i) {
  asm volatile("bar.sync %0, 64;" ::"r"(1 + (i >> 5)) : "memory");
}

// own half of the pair's summed partial spinors (thread (hf, i) stores the
// part its partner owns in slot hf and reads its partner's slot 1 - hf).  Only
// the pair's two warps meet here; every caller passes a CTA-wide barrier
// before its next call, so no slot is overwritten before the partner read it.
template <typename T>
__device__ __forceinline__ Half<T> pair_reduce_s(const Spinor<T>& acc, int hf, int i, int np, T* xb) {
  s_half_store(xb, np, i, hf, half_of(acc, 1 - hf));
  pair_warps_sync(i);
  return half_axpy(half_of(acc, hf), s_half(xb, np, i, 1 - hf), T(1));
}

// full spinor from the owned halves of a pair (ends with a barrier, so the
// buffer can be reused at once)
template <typename T>
__device__ __forceinline__ Spinor<T> pair_full_s(const Half<T>& own, int hf, int i, int np, T* xb) {
  s_half_store(xb, np, i, hf, own);
  __syncthreads();
  const Half<T> o = s_half(xb, np, i, 1 - hf);
  __syncthreads();
  Spinor<T> v;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v.c[s][c] = hf ? o.c[s][c] : own.c[s][c];
      v.c[2 + s][c] = hf ? own.c[s][c] : o.c[s][c];
    }
  return v;
}

// owned half of -1/2 (sum of hops) at site r
template <typename T, typename ST>
__device__ __forceinline__ Half<T> block_hops(const ST& st, int n, int r, const T* src, const int pk[2], int off,
                                              int hf, int i, int np, T* xb) {
  Half<T> h = pair_reduce_s(hops_pair<T>(st, n, r, src, pk, off, hf), hf, i, np, xb);
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) h.c[s][c] = T(-0.5) * h.c[s][c];
  return h;
}

// deterministic CTA-wide sum of 3 values; every thread gets the totals.  The
// caller must pass another barrier before the next call.
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
  // lane k of every warp takes warp k's partial sums; a butterfly over the
  // lanes leaves every thread the totals, summed in the same order everywhere
  const int l = threadIdx.x & 31;
  a = l < nw ? red[3 * l] : T(0);
  b = l < nw ? red[3 * l + 1] : T(0);
  c = l < nw ? red[3 * l + 2] : T(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  // no closing barrier: red is written again only after later barriers
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

// FP64 values into the arithmetic type and back (integer-pipe conversions)
__device__ __forceinline__ void from_f64(double x, float& y) { y = f64_to_f32(x); }
__device__ __forceinline__ void from_f64(double x, double& y) { y = x; }
__device__ __forceinline__ double as_f64(float x) { return f32_to_f64(x); }
__device__ __forceinline__ double as_f64(double x) { return x; }

// owned half of an FP32 / FP64 spinor field in global memory (spins 2 hf, 2 hf + 1
// are reals 12 hf .. 12 hf + 11: float4 chunks 3 hf .. 3 hf + 2, or double2 chunks 6 hf ..)
template <int PS, typename T>
__device__ __forceinline__ Half<T> g_half(const FieldPtr& f, int Vb, int blk, int r, int hf) {
  Half<T> h;
  if constexpr (PS == P64) {
    const double2* d = (const double2*)f.data + ((long long)blk * 12 + 6 * hf) * Vb + r;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double2 v = d[(long long)k * Vb];
      from_f64(v.x, h.c[k / 3][k % 3].re);
      from_f64(v.y, h.c[k / 3][k % 3].im);
    }
  } else {
    const float4* d = (const float4*)f.data + ((long long)blk * 6 + 3 * hf) * Vb + r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 v = d[(long long)k * Vb];
      h.c[(2 * k) / 3][(2 * k) % 3] = {(T)v.x, (T)v.y};
      h.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = {(T)v.z, (T)v.w};
    }
  }
  return h;
}

template <int PS, typename T>
__device__ __forceinline__ void g_half_store(const FieldPtr& f, int Vb, int blk, int r, int hf, const Half<T>& h) {
  if constexpr (PS == P64) {
    double2* d = (double2*)f.data + ((long long)blk * 12 + 6 * hf) * Vb + r;
#pragma unroll
    for (int k = 0; k < 6; ++k) d[(long long)k * Vb] = make_double2(as_f64(h.c[k / 3][k % 3].re), as_f64(h.c[k / 3][k % 3].im));
  } else {
    float4* d = (float4*)f.data + ((long long)blk * 6 + 3 * hf) * Vb + r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const cpx<T> a = h.c[(2 * k) / 3][(2 * k) % 3], b = h.c[(2 * k + 1) / 3][(2 * k + 1) % 3];
      d[(long long)k * Vb] = make_float4((float)a.re, (float)a.im, (float)b.re, (float)b.im);
    }
  }
}

// owned half of a double-float spinor field (the FP64 layout with float4
// chunks (re hi, re lo, im hi, im lo)): the high parts, i.e. the values
// rounded to FP32 -- what the block solver computes with
template <typename T>
__device__ __forceinline__ Half<T> g_half_df(const FieldPtr& f, int Vb, int blk, int r, int hf) {
  Half<T> h;
  const float4* d = (const float4*)f.data + ((long long)blk * 12 + 6 * hf) * Vb + r;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = d[(long long)k * Vb];
    if constexpr (sizeof(T) == 8)
      h.c[k / 3][k % 3] = {f32_to_f64(v.x) + f32_to_f64(v.y), f32_to_f64(v.z) + f32_to_f64(v.w)};
    else
      h.c[k / 3][k % 3] = {v.x, v.z};
  }
  return h;
}

// store an owned half into a double-float field: FP32 values are exact high
// parts (low parts 0); FP64 values are split
template <typename T>
__device__ __forceinline__ void g_half_store_df(const FieldPtr& f, int Vb, int blk, int r, int hf, const Half<T>& h) {
  float4* d = (float4*)f.data + ((long long)blk * 12 + 6 * hf) * Vb + r;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const cpx<T> v = h.c[k / 3][k % 3];
    if constexpr (sizeof(T) == 8) {
      const df a = df_from_f64(v.re), b = df_from_f64(v.im);
      d[(long long)k * Vb] = make_float4(a.hi, a.lo, b.hi, b.lo);
    } else {
      d[(long long)k * Vb] = make_float4(v.re, 0.f, v.im, 0.f);
    }
  }
}

// owned half of a 16-bit spinor record ([blk][3 chunks][Vb] uint4 of 8 reals,
// complex k at chunk k / 4): half hf is chunk 2 hf and the hf-th 8-byte half of
// chunk 1, scaled by the site's norm
template <int P>
__device__ __forceinline__ Half<float> g_half16(const FieldPtr& f, int Vb, int blk, int r, int hf) {
  const uint4* d = (const uint4*)f.data + (long long)blk * 3 * Vb + r;
  const uint4 a = __ldg(d + (long long)(2 * hf) * Vb);
  const uint2 b = __ldg((const uint2*)(d + Vb) + hf);
  const float s = f.norm ? __ldg(f.norm + (long long)blk * Vb + r) : 1.0f;
  // complexes 6 hf .. 6 hf + 5: hf = 0 -> chunk 0 (0-3), chunk 1 low (4-5);
  // hf = 1 -> chunk 1 high (6-7), chunk 2 (8-11)
  const uint32_t w[6] = {hf ? b.x : a.x, hf ? b.y : a.y, hf ? a.x : a.z, hf ? a.y : a.w, hf ? a.z : b.x, hf ? a.w : b.y};
  Half<float> h;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 x = to_f2<P>(w[k]);
    h.c[k / 3][k % 3] = {s * x.x, s * x.y};
  }
  return h;
}

// receive the other colour's face contributions at site (blk, r) for the
// directions of this thread; returns a partial full spinor.  A site lies on at
// most one face per direction (block extents are at least 2), so one read per
// direction serves both kinds of face, and a warp waits for one read per
// direction however its sites split between the kinds.
template <typename T, typename ST>
__device__ __forceinline__ Spinor<T> receive_faces(const SapArgs& a, const void* faces, const ST& st, int blk, int r,
                                                   const int y[4], const int n[4], int hf) {
  const Geom& g = a.g;
  Spinor<T> acc;
  zero(acc);
#pragma unroll 1
  for (int m = 0; m < 2; ++m) {
    const int mu = 2 * hf + m;
    const SpinDir<T> d = spin_dir<T>(mu);
    const int ymu = mu == 0 ? y[0] : (mu == 1 ? y[1] : (mu == 2 ? y[2] : y[3]));
    const int nmu = mu == 0 ? n[0] : (mu == 1 ? n[1] : (mu == 2 ? n[2] : n[3]));
    // up: from block + mu, U_mu(y) (1 - g) part, projected by the sender;
    // down: from block - mu, U^+ (1 + g) part, multiplied by the sender
    const bool up = ymu == g.b[mu] - 1, down = ymu == 0;
    if (!up && !down) continue;
    const int nbk = up ? (nmu + 1 < g.nb[mu] ? blk + g.bstr[mu] : blk - (g.nb[mu] - 1) * g.bstr[mu])
                       : (nmu > 0 ? blk - g.bstr[mu] : blk + (g.nb[mu] - 1) * g.bstr[mu]);
    const Half<T> h = face_load<T>(a, faces, nbk, up ? 2 * mu : 2 * mu + 1, face_index(g, y, mu));
    if (up)
      expand_add_rt<-1>(acc, umul(st.link(r, mu), h), T(1), d);
    else
      expand_add_rt<+1>(acc, h, T(1), d);
  }
  return acc;
}

// write the face contributions of the correction chi at site (blk, r) for the
// directions of this thread
template <typename T, typename ST>
__device__ __forceinline__ void send_faces(const SapArgs& a, void* faces, const ST& st, int blk, int r,
                                           const int y[4], const int n[4], const Spinor<T>& chi, int hf) {
  const Geom& g = a.g;
#pragma unroll 1
  for (int m = 0; m < 2; ++m) {
    const int mu = 2 * hf + m;
    const SpinDir<T> d = spin_dir<T>(mu);
    const int ymu = mu == 0 ? y[0] : (mu == 1 ? y[1] : (mu == 2 ? y[2] : y[3]));
    const int nmu = mu == 0 ? n[0] : (mu == 1 ? n[1] : (mu == 2 ? n[2] : n[3]));
    if (ymu == 0) {  // to y = x - mu: 1/2 eta_mu(y) (1 - g) chi, projected
      const T f = T(0.5) * ((nmu == 0) ? bc_of<T>(g, mu) : T(1));
      Half<T> h = project_rt<-1>(chi, d);
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) h.c[s][c] = f * h.c[s][c];
      face_store<T>(a, faces, blk, 2 * mu, face_index(g, y, mu), h);
    }
    if (ymu == g.b[mu] - 1) {  // to y = x + mu: 1/2 eta_mu(x) U_mu(x)^+ (1 + g) chi, projected
      const T f = T(0.5) * ((nmu == g.nb[mu] - 1) ? bc_of<T>(g, mu) : T(1));
      Half<T> w = udmul(st.link(r, mu), project_rt<+1>(chi, d));
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) w.c[s][c] = f * w.c[s][c];
      face_store<T>(a, faces, blk, 2 * mu + 1, face_index(g, y, mu), w);
    }
  }
}

template <int P>
struct StageFor {
  typedef HalfExpStage<P> type;
};
template <>
struct StageFor<P32> {
  typedef ExpandedStage<float> type;
};
template <>
struct StageFor<P64> {
  typedef ExpandedStage<double> type;
};

// site pairs per half-CTA: Vbh rounded up to whole warps
__host__ __device__ __forceinline__ int pairs_per_half(int Vbh) { return (Vbh + 31) / 32 * 32; }

// VB: the block volume as a compile-time constant (shared-memory and link
// offsets become immediates, which frees registers), or 0 for any volume
// TILED: the CTA solves a tile of right-hand sides (the loop below runs over
// them); otherwise exactly one, right-hand side 0, and the loop folds away
template <int P, typename T, int VB, bool TILED>
__global__ void __launch_bounds__(512) sap_sweep_kernel(SapArgs a) {
  typedef typename StageFor<P>::type ST;
  constexpr bool kHalf = (P == P16 || P == PB16);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Geom& g = a.g;
  const int Vb = VB ? VB : g.Vb, Vbh = VB ? VB / 2 : g.Vbh;
  const int np = pairs_per_half(Vbh);

  // shared memory: staged block fields, then the FP vectors r (even sites),
  // t (odd sites), the pair-exchange buffer, the reduction scratch and the
  // staging barrier.  With 16-bit fields the compressed links land in the
  // vector area first and are expanded into the link area.
  ST st;
  const size_t stage_bytes = ST::bytes(Vb);
  st.base_init(smem_raw, Vb);
  const int ns = Vbh + 1;  // stride of the chunked fields r and t; slot Vbh is a zero site
  T* s_r = (T*)(smem_raw + stage_bytes);
  T* s_t = s_r + 24 * ns;
  T* s_x = s_t + 24 * ns;  // pair exchange: 24 reals x np, chunked
  T* s_red = s_x + 24 * np;
  uint64_t* bar = (uint64_t*)(s_red + 3 * 32);

  // block of the requested colour: pairs (2k, 2k+1) differ in n3 only, hence in colour
  int blk = 2 * blockIdx.x;
  int n[4];
  block_coords(g, blk, n);
  if (((n[0] + n[1] + n[2] + n[3]) & 1) != a.colour) {
    ++blk;
    ++n[3];
  }

  // right-hand sides of this CTA; a tile with none to solve stages nothing
  const int rhs0 = TILED ? blockIdx.y * a.rt : 0, rhs1 = TILED ? min(rhs0 + a.rt, a.nrhs) : 1;
  if (TILED) {
    bool any = false;
    for (int rr = rhs0; rr < rhs1; ++rr) any |= (a.mask == nullptr || a.mask[rr] != 0);
    if (!any) return;
  }

  // ---- stage the block's links and clover (once for the whole tile)
  if constexpr (kHalf) {
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();  // every thread sees the initialised barrier before it waits on it
    if (threadIdx.x < 32) stage_issue<P>(a, blk, (unsigned char*)s_r, (unsigned char*)st.base + 144 * Vb, bar);
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

  // site pair i owns even site i and odd site Vbh + i; thread half hf (uniform
  // across a warp) holds spin components 2 hf, 2 hf + 1 and computes the hops
  // in directions 2 hf, 2 hf + 1.  Pairs with i >= Vbh (blocks of fewer than
  // 64 sites) compute on site 0 and store nothing.
  const int hf = threadIdx.x / np, i = threadIdx.x - hf * np;
  const bool act = i < Vbh;
  const int re = act ? i : 0, ro = Vbh + re;

  // ---- in-block neighbour tables of the two sites, own directions only.
  // In-block lexicographic sites 2m and 2m + 1 differ only in y3 (b3 is even),
  // hence in parity, so a site's rank among its parity is j >> 1: no table.
  int ye[4], yo[4];
  {
    const int pe = __ldg(g.r2y + re), po = __ldg(g.r2y + ro);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      ye[mu] = ycoord(pe, mu);
      yo[mu] = ycoord(po, mu);
    }
  }
  int pkE[2], pkO[2];  // even site: indices into t (site - Vbh); odd site: into r (= site); Vbh = absent
  {
    const int je = ye[0] * g.ystr[0] + ye[1] * g.ystr[1] + ye[2] * g.ystr[2] + ye[3] * g.ystr[3];
    const int jo = yo[0] * g.ystr[0] + yo[1] * g.ystr[1] + yo[2] * g.ystr[2] + yo[3] * g.ystr[3];
    int pke[4], pko[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int ef = ye[mu] + 1 < g.b[mu] ? (je + g.ystr[mu]) >> 1 : Vbh;
      const int eb = ye[mu] > 0 ? (je - g.ystr[mu]) >> 1 : Vbh;
      const int of = yo[mu] + 1 < g.b[mu] ? (jo + g.ystr[mu]) >> 1 : Vbh;
      const int ob = yo[mu] > 0 ? (jo - g.ystr[mu]) >> 1 : Vbh;
      pke[mu] = ef | (eb << 16);
      pko[mu] = of | (ob << 16);
    }
    pkE[0] = hf ? pke[2] : pke[0];
    pkE[1] = hf ? pke[3] : pke[1];
    pkO[0] = hf ? pko[2] : pko[0];
    pkO[1] = hf ? pko[3] : pko[1];
  }

  bool staged = false;
#pragma unroll 1
  for (int rr = rhs0; rr < rhs1; ++rr) {
    if (TILED && a.mask != nullptr && a.mask[rr] == 0) continue;  // uniform across the CTA
    if (threadIdx.x >= 32 && threadIdx.x < 64)
      prefetch_late_reads<T, PsiPrec<P>::value>(a, rhs_faces(a, rr), rhs_psi(a, rr), blk, n);

    // ---- residual of the two sites (own halves only: the pair's two threads
    // read complementary halves)
    Half<T> rho_e, rho_o;
    if (a.read_eta && a.io32) {
      const Half<float> de = g_half<P32, float>(rhs_eta(a, rr), Vb, blk, re, hf);
      const Half<float> dd = g_half<P32, float>(rhs_eta(a, rr), Vb, blk, ro, hf);
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          rho_e.c[s][c] = {(T)de.c[s][c].re, (T)de.c[s][c].im};
          rho_o.c[s][c] = {(T)dd.c[s][c].re, (T)dd.c[s][c].im};
        }
    } else if (a.read_eta && a.io_df) {
      rho_e = g_half_df<T>(rhs_eta(a, rr), Vb, blk, re, hf);
      rho_o = g_half_df<T>(rhs_eta(a, rr), Vb, blk, ro, hf);
    } else if (a.read_eta) {
      rho_e = g_half<P64, T>(rhs_eta(a, rr), Vb, blk, re, hf);
      rho_o = g_half<P64, T>(rhs_eta(a, rr), Vb, blk, ro, hf);
    } else if constexpr (kHalf) {
      rho_e = g_half16<P>(rhs_rho(a, rr), Vb, blk, re, hf);
      rho_o = g_half16<P>(rhs_rho(a, rr), Vb, blk, ro, hf);
    } else {
      rho_e = g_half<P, T>(rhs_rho(a, rr), Vb, blk, re, hf);
      rho_o = g_half<P, T>(rhs_rho(a, rr), Vb, blk, ro, hf);
    }
    if (!staged) {
      if constexpr (kHalf) {
        // every thread waits (bounded) for the staging copies; a time-out is made
        // block-uniform, recorded, and the block is skipped
        const bool ok = mbar_wait_bounded(bar, a.wait_cycles);
        if (__syncthreads_or(!ok)) {
          if (threadIdx.x == 0) atomicExch(a.err, 1);
          mbar_wait_bounded(bar, kWaitCycles);  // let copies still in flight land before the CTA exits
          return;
        }
        expand_links<P>((const unsigned char*)s_r, (unsigned char*)st.base, Vb);
      }
      __syncthreads();
      {  // zero sites of r and t (the 16-bit links' landing zone is consumed by now)
        typedef typename Chunk<T>::type C;
        constexpr int NCH = 24 / Chunk<T>::R;
        if (threadIdx.x < 2 * NCH) {
          const T z[Chunk<T>::R] = {};
          C* base = (C*)(threadIdx.x < NCH ? s_r : s_t);
          base[(threadIdx.x % NCH) * ns + Vbh] = chunk_make(z);
        }
      }
      staged = true;
    }
    if (TILED) __syncthreads();  // the previous right-hand side's last reads of r, t and the exchange buffer are done
    if (a.faces_in) {
      rho_e = half_axpy(rho_e, pair_reduce_s(receive_faces<T>(a, rhs_faces(a, rr), st, blk, re, ye, n, hf), hf, i, np, s_x),
                        T(1));
      __syncthreads();
      rho_o = half_axpy(rho_o, pair_reduce_s(receive_faces<T>(a, rhs_faces(a, rr), st, blk, ro, yo, n, hf), hf, i, np, s_x),
                        T(1));
    }
    // etahat = rho_e - D_eo A_oo^-1 rho_o: first t = A_oo^-1 rho_o
    if (act) s_half_store(s_t, ns, i, hf, clover_half(st, ro, hf, rho_o));
    __syncthreads();
    Half<T> r = half_axpy(rho_e, block_hops<T>(st, ns, re, s_t, pkE, Vbh, hf, i, np, s_x), T(-1));
    Half<T> x;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) x.c[s][c] = {T(0), T(0)};
    if (act) s_half_store(s_r, ns, i, hf, r);
    __syncthreads();

    // ---- MR on Dhat = A_ee - D_eo A_oo^-1 D_oe, x_e = 0, r = etahat.  Each
    // step runs two phases through one code path: phase 0 (odd sites)
    // t = A_oo^-1 D_oe r, phase 1 (even sites) p = A_ee r - D_eo t.
#pragma unroll 1
    for (int step = 0; step < 2 * a.nmr; ++step) {
      const int ph = step & 1;
      const int pk2[2] = {ph ? pkE[0] : pkO[0], ph ? pkE[1] : pkO[1]};
      const Half<T> hq = block_hops<T>(st, ns, ph ? re : ro, ph ? s_t : s_r, pk2, ph ? Vbh : 0, hf, i, np, s_x);
      const Half<T> cl = clover_half(st, ph ? re : ro, hf, ph ? r : hq);
      if (ph == 0) {
        if (act) s_half_store(s_t, ns, i, hf, cl);
        __syncthreads();
        continue;
      }
      const Half<T> p = half_axpy(cl, hq, T(-1));
      T pr_re = 0, pr_im = 0, pp = 0;
      if (act) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const cpx<T> v = p.c[s][c], w = r.c[s][c];
            pr_re += v.re * w.re + v.im * w.im;
            pr_im += v.re * w.im - v.im * w.re;
            pp += v.re * v.re + v.im * v.im;
          }
      }
      cta_sum3(pr_re, pr_im, pp, s_red);
      const T inv = pp > T(0) ? T(1) / pp : T(0);
      const cpx<T> alpha = {pr_re * inv, pr_im * inv};
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          x.c[s][c] = cmadd(alpha, r.c[s][c], x.c[s][c]);
          r.c[s][c] = r.c[s][c] - cmul(alpha, p.c[s][c]);
        }
      if (act) s_half_store(s_r, ns, i, hf, r);
      __syncthreads();
    }

    // ---- chi_o = A_oo^-1 (rho_o - D_oe chi_e)
    if (act) s_half_store(s_r, ns, i, hf, x);
    __syncthreads();
    const Half<T> chi_o =
        clover_half(st, ro, hf, half_axpy(rho_o, block_hops<T>(st, ns, ro, s_r, pkO, 0, hf, i, np, s_x), T(-1)));
    __syncthreads();

    // ---- outputs: solution, block residual (r on even, 0 on odd), faces
    constexpr int PS = PsiPrec<P>::value;
    typedef typename std::conditional<PS == P64, double, float>::type TS;
    const Spinor<T> x_full = pair_full_s(x, hf, i, np, s_x);
    const Spinor<T> chio_full = pair_full_s(chi_o, hf, i, np, s_x);
    const Spinor<T> r_full = pair_full_s(r, hf, i, np, s_x);
    if (act) {
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const int rs = half ? ro : re;
        const Half<T>& chi = half ? chi_o : x;
        Half<TS> v;
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) v.c[s][c] = {(TS)chi.c[s][c].re, (TS)chi.c[s][c].im};
        if (a.psi_mode == 1 || a.psi_mode == 3) v = half_axpy(v, g_half<PS, TS>(rhs_psi(a, rr), Vb, blk, rs, hf), TS(1));
        if (a.psi_mode <= 1) {
          g_half_store<PS, TS>(rhs_psi(a, rr), Vb, blk, rs, hf, v);
        } else if (a.io_df && !a.out32) {
          g_half_store_df<TS>(rhs_out(a, rr), Vb, blk, rs, hf, v);
        } else if (a.io32 || a.out32) {
          Half<float> fv;
#pragma unroll
          for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) fv.c[s][c] = {(float)v.c[s][c].re, (float)v.c[s][c].im};
          g_half_store<P32, float>(rhs_out(a, rr), Vb, blk, rs, hf, fv);
        } else {
          g_half_store<P64, TS>(rhs_out(a, rr), Vb, blk, rs, hf, v);  // widened on the integer pipes
        }
      }
      if (a.write_rho && hf == 0) {
        store_spinor<P, T>(rhs_rho(a, rr), Vb, blk, re, r_full);
        Spinor<T> z;
        zero(z);
        store_spinor<P, T>(rhs_rho(a, rr), Vb, blk, ro, z);
      }
      if (a.faces_out) {
        // the coordinates again (cheaper than keeping 12 registers through the MR steps)
        int n2[4], ye2[4], yo2[4];
        block_coords(g, blk, n2);
        const int pe = g.r2y[re], po = g.r2y[ro];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          ye2[mu] = ycoord(pe, mu);
          yo2[mu] = ycoord(po, mu);
        }
        send_faces<T>(a, rhs_faces(a, rr), st, blk, re, ye2, n2, x_full, hf);
        send_faces<T>(a, rhs_faces(a, rr), st, blk, ro, yo2, n2, chio_full, hf);
      }
    }
  }
}

template <int P, typename T>
static size_t sap_smem_bytes(const Geom& g) {
  typedef typename StageFor<P>::type ST;
  const int np = pairs_per_half(g.Vbh);
  return ST::bytes(g.Vb) + sizeof(T) * (2 * 24 * (size_t)(g.Vbh + 1) + 24 * (size_t)np + 3 * 32) + 16;
}

// block volumes with their own instantiation (4^4 and 8 x 4^3 blocks)
static int sap_vb_key(int Vb) { return Vb == 256 || Vb == 512 ? Vb : 0; }

template <int P, typename T, int VB>
static int set_smem_attr_vb(size_t smem) {
  QCD_CUDA(cudaFuncSetAttribute(sap_sweep_kernel<P, T, VB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  QCD_CUDA(cudaFuncSetAttribute(sap_sweep_kernel<P, T, VB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  return QCD_OK;
}

template <int P, typename T>
static int set_smem_attr(const Geom& g, int maxsm) {
  const size_t smem = sap_smem_bytes<P, T>(g);
  if (smem > (size_t)maxsm) return QCD_ERR_UNSUPPORTED;
  if constexpr (P == P16 || P == PB16) {
    if (sap_vb_key(g.Vb) == 256) return set_smem_attr_vb<P, T, 256>(smem);
    if (sap_vb_key(g.Vb) == 512) return set_smem_attr_vb<P, T, 512>(smem);
  }
  return set_smem_attr_vb<P, T, 0>(smem);
}

template <int P, typename T, int VB>
static void sap_launch_vb(dim3 grid, int threads, size_t smem, cudaStream_t s, const SapArgs& a) {
  if (a.nrhs > 1 || a.mask)
    sap_sweep_kernel<P, T, VB, true><<<grid, threads, smem, s>>>(a);
  else
    sap_sweep_kernel<P, T, VB, false><<<grid, threads, smem, s>>>(a);
}

// launch one colour half-sweep; 16-bit block fields of 4^4 and 8 x 4^3 blocks
// run the instantiation for their volume, single right-hand sides the
// untiled one
template <int P, typename T>
static void sap_launch(const Geom& g, dim3 grid, int threads, cudaStream_t s, const SapArgs& a) {
  const size_t smem = sap_smem_bytes<P, T>(g);
  if constexpr (P == P16 || P == PB16) {
    if (sap_vb_key(g.Vb) == 256) return sap_launch_vb<P, T, 256>(grid, threads, smem, s, a);
    if (sap_vb_key(g.Vb) == 512) return sap_launch_vb<P, T, 512>(grid, threads, smem, s, a);
  }
  sap_launch_vb<P, T, 0>(grid, threads, smem, s, a);
}

// allocate the SAP work fields for nr right-hand sides and set the kernel's
// shared-memory limit for this geometry (outside any stream capture)
int sap_prepare(qcd_ctx* c, SapWork& w, int prec, cudaStream_t s, int nr) {
  const Geom& g = c->g;
  if (prec < P64 || prec > PB16 || nr < 1) return QCD_ERR_ARG;
  if (g.Vbh > 256) return QCD_ERR_UNSUPPORTED;
  QCD_TRY(ensure_gauge(c, prec, s));
  QCD_TRY(ensure_clover(c, prec, s));
  int dev = 0, maxsm = 0;
  QCD_CUDA(cudaGetDevice(&dev));
  QCD_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  switch (prec) {
    case P64: QCD_TRY((set_smem_attr<P64, double>(g, maxsm))); break;
    case P32: QCD_TRY((set_smem_attr<P32, float>(g, maxsm))); break;
    case P16: QCD_TRY((set_smem_attr<P16, float>(g, maxsm))); break;
    default: QCD_TRY((set_smem_attr<PB16, float>(g, maxsm))); break;
  }
  if (w.prec == prec && w.nr == nr) return QCD_OK;
  const bool dbl = prec == P64;
  rec_free(w.rho);
  rec_free(w.psi);
  if (w.faces) cudaFree(w.faces);
  w.faces = nullptr;
  w.prec = -1;
  w.nr = 0;
  QCD_TRY(rec_alloc(w.rho, prec, 24, c->V * nr));
  QCD_TRY(rec_alloc(w.psi, dbl ? P64 : P32, 24, c->V * nr));
  int F = 0;
  for (int mu = 0; mu < 4; ++mu) F += 2 * (g.Vb / g.b[mu]);
  w.faces_bytes = (size_t)c->nblk * F * 12 * (dbl ? 8 : 4) * nr;
  if (cudaMalloc(&w.faces, w.faces_bytes) != cudaSuccess) {
    cudaGetLastError();
    w.faces = nullptr;
    return QCD_ERR_NOMEM;
  }
  w.prec = prec;
  w.nr = nr;
  return QCD_OK;
}

// right-hand sides per CTA of the SAP launch: the context's tuned value, else
// the largest tile that still gives every SM four CTAs of work per launch
int sap_tile(qcd_ctx* c, int nr) {
  if (nr <= 1) return 1;
  if (c->sap_rt > 0) return c->sap_rt < nr ? c->sap_rt : nr;
  const long long per_rhs = c->nblk / 2;
  int rt = 1;
  while (rt < nr && per_rhs * ((nr + 2 * rt - 1) / (2 * rt)) >= 4 * 152) rt *= 2;
  return rt;
}

// psi = M_SAP eta (both FP64 or both FP32 fields) for every right-hand side of
// B (fields V sites apart; B.mask skips right-hand sides); allocates nothing
// once sap_prepare ran for prec and B.n
int sap_apply(qcd_ctx* c, SapWork& w, const Rec& eta64, const Rec& psi64, int ncy, int nmr, int prec,
              cudaStream_t s, const Batch& B, int rt) {
  const Geom& g = c->g;
  // a double-float source with a double-float or an FP32 result (FP32 holds the
  // FP32 block solution exactly)
  const bool df_in = eta64.prec == PDF && (psi64.prec == PDF || psi64.prec == P32);
  if (!df_in && (eta64.prec != psi64.prec || (eta64.prec != P64 && eta64.prec != P32))) return QCD_ERR_ARG;
  if (ncy < 1 || nmr < 0 || B.n < 1) return QCD_ERR_ARG;
  if (w.prec != prec || w.nr != B.n) QCD_TRY(sap_prepare(c, w, prec, s, B.n));
  if (rt < 1) rt = sap_tile(c, B.n);
  const bool dbl = prec == P64;
  SapArgs a;
  a.g = g;
  a.nmr = nmr;
  a.U = c->U[prec];
  a.Ahat = c->Ahat[prec].ptr();
  a.io32 = eta64.prec == P32;
  a.io_df = df_in;
  a.out32 = df_in && psi64.prec == P32;
  a.eta = eta64.ptr();
  a.rho = w.rho.ptr();
  a.psi = w.psi.ptr();
  a.out = psi64.ptr();
  a.faces = w.faces;
  a.err = (int*)(c->d_scalars + 128);
  a.wait_cycles = c->dbg_sap_wait_cycles;
  a.extra_tx = c->dbg_sap_extra_tx;
  int off = 0;
  for (int mu = 0; mu < 4; ++mu) {
    a.fo[2 * mu] = off;
    off += g.Vb / g.b[mu];
    a.fo[2 * mu + 1] = off;
    off += g.Vb / g.b[mu];
  }
  a.F = off;
  a.nrhs = B.n;
  a.rt = rt;
  a.mask = B.mask;
  a.eta_rs = (long long)c->V * (a.io32 ? 96 : 192);  // FP64 and double-float fields: 192 B per site
  a.out_rs = (long long)c->V * (a.io32 || a.out32 ? 96 : 192);
  a.rho_rs = (long long)c->V * chunks(prec, 24) * 16;
  a.rho_ns = w.rho.norm ? c->V : 0;
  a.psi_rs = (long long)c->V * (dbl ? 192 : 96);
  a.faces_rs = (long long)c->nblk * a.F * 12 * (dbl ? 8 : 4);
  const dim3 grid((unsigned)(c->nblk / 2), (unsigned)((B.n + rt - 1) / rt));
  const int threads = 2 * pairs_per_half(g.Vbh);  // two threads per site pair, halves warp-aligned
  // flops (the 1320 + 504 convention): per solved site the Schur operator
  // costs about one D per MR step, plus about one more D for the source and
  // the back-substitution
  const double flops = (double)(nmr + 1) * 1824.0 * (double)c->V / 2.0 * B.n;
  const double sb = dbl ? 8 : (prec == P32 ? 4 : 2);
  // algorithmic bytes: links and clover of the solved blocks once per tile,
  // residual and solution in and out per right-hand side
  const double tiles = (double)((B.n + rt - 1) / rt);
  const double bytes = (double)c->V / 2 *
                       ((4 * (dbl ? 18 : 12) * sb + 72 * sb) * tiles + (2 * 24 * sb + 2 * 24 * (dbl ? 8 : 4)) * B.n);
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
      switch (prec) {
        case P64: sap_launch<P64, double>(g, grid, threads, s, a); break;
        case P32: sap_launch<P32, float>(g, grid, threads, s, a); break;
        case P16: sap_launch<P16, float>(g, grid, threads, s, a); break;
        case PB16: sap_launch<PB16, float>(g, grid, threads, s, a); break;
        default: return QCD_ERR_ARG;
      }
      QCD_LAUNCHED();
    }
  return QCD_OK;
}

}  // namespace qcd
