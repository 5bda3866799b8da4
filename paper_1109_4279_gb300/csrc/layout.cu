// Block-major even/odd layout (Sec. 5), spinor import/export, gauge-field
// upload, SU(3) check and reduced-precision link compression.
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace qcd {

int setup_geometry(qcd_ctx* c) {
  Geom& g = c->g;
  long long V = 1;
  int Vb = 1, nblk = 1;
  for (int mu = 0; mu < 4; ++mu) {
    int L = c->p.dims[mu], b = c->p.block[mu];
    if (L <= 0 || b <= 0) return QCD_ERR_ARG;
    if (b % 2 || L % b || (L / b) % 2 || b > 64) return QCD_ERR_GEOMETRY;
    g.L[mu] = L;
    g.b[mu] = b;
    g.nb[mu] = L / b;
    g.bc[mu] = c->p.bc[mu];
    g.bcf[mu] = (float)c->p.bc[mu];
    V *= L;
    Vb *= b;
    nblk *= L / b;
  }
  if (Vb > 4096) return QCD_ERR_GEOMETRY;
  g.bstr[3] = 1;
  g.ystr[3] = 1;
  for (int mu = 2; mu >= 0; --mu) {
    g.bstr[mu] = g.bstr[mu + 1] * g.nb[mu + 1];
    g.ystr[mu] = g.ystr[mu + 1] * g.b[mu + 1];
  }
  g.Vb = Vb;
  g.Vbh = Vb / 2;
  g.nblk = nblk;
  g.V = V;
  c->V = V;
  c->nblk = nblk;

  // r <-> local coordinates.  b3 even: sites j and j ^ 1 differ only in y3,
  // hence in parity, so (parity, j >> 1) enumerates each parity exactly once.
  std::vector<int> tab(2 * Vb);
  int* r2y = tab.data();
  int* j2r = tab.data() + Vb;
  for (int j = 0; j < Vb; ++j) {
    int y[4], t = j;
    for (int mu = 3; mu >= 0; --mu) {
      y[mu] = t % g.b[mu];
      t /= g.b[mu];
    }
    int par = (y[0] + y[1] + y[2] + y[3]) & 1;
    int r = par * g.Vbh + (j >> 1);
    j2r[j] = r;
    r2y[r] = y[0] | (y[1] << 8) | (y[2] << 16) | (y[3] << 24);
  }
  QCD_CUDA(cudaMalloc(&c->d_tables, sizeof(int) * 2 * Vb));
  QCD_CUDA(cudaMemcpy(c->d_tables, tab.data(), sizeof(int) * 2 * Vb, cudaMemcpyHostToDevice));
  g.r2y = c->d_tables;
  g.j2r = c->d_tables + Vb;
  return QCD_OK;
}

// ------------------------------------------------------------------------
// spinor import / export: lexicographic (V, 4, 3) complex128 <-> internal
// ------------------------------------------------------------------------
// sites [s0, s1) of the internal order (whole blocks: a range of blocks)
template <int P>
__global__ void import_kernel(Geom g, const double* __restrict__ lex, FieldPtr out, long long field_stride_sites,
                              long long s0, long long s1) {
  long long s = s0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= s1) return;
  const int rhs = blockIdx.y;
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  int x[4];
  global_coords(g, blk, r, x);
  const double2* src = (const double2*)lex + ((long long)rhs * g.V + lex_index(g, x)) * 12;
  double v[24];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 d = __ldg(src + k);
    v[2 * k] = d.x;
    v[2 * k + 1] = d.y;
  }
  FieldPtr f = out;
  const int NC = (P == P64 || P == PDF) ? 12 : (P == P32 ? 6 : 3);
  f.data = (char*)out.data + (size_t)rhs * field_stride_sites * NC * 16;
  if (out.norm) f.norm = out.norm + (size_t)rhs * field_stride_sites;
  if constexpr (P == P64 || P == PDF) {
    store_record<P, 24, double>(f, g.Vb, blk, r, v);
  } else {
    float w[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) w[k] = f64_to_f32(v[k]);
    store_record<P, 24, float>(f, g.Vb, blk, r, w);
  }
}

template <int P>
__global__ void export_kernel(Geom g, FieldPtr in, double* __restrict__ lex, long long field_stride_sites,
                              long long s0, long long s1) {
  long long s = s0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= s1) return;
  const int rhs = blockIdx.y;
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  int x[4];
  global_coords(g, blk, r, x);
  FieldPtr f = in;
  const int NC = (P == P64 || P == PDF) ? 12 : (P == P32 ? 6 : 3);
  f.data = (char*)in.data + (size_t)rhs * field_stride_sites * NC * 16;
  if (in.norm) f.norm = in.norm + (size_t)rhs * field_stride_sites;
  double v[24];
  if constexpr (P == P64 || P == PDF) {
    load_record<P, 24, double>(f, g.Vb, blk, r, v);
  } else {
    float w[24];
    load_record<P, 24, float>(f, g.Vb, blk, r, w);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = f32_to_f64(w[k]);
  }
  double2* dst = (double2*)lex + ((long long)rhs * g.V + lex_index(g, x)) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = make_double2(v[2 * k], v[2 * k + 1]);
}

static int import_range(qcd_ctx* c, const double* lex, const Rec& out, int nrhs, long long s0, long long s1,
                        cudaStream_t s) {
  if (out.nreal != 24) return QCD_ERR_ARG;
  if (s1 <= s0) return QCD_OK;
  dim3 grid((unsigned)((s1 - s0 + 255) / 256), nrhs);
  switch (out.prec) {
    case P64: import_kernel<P64><<<grid, 256, 0, s>>>(c->g, lex, out.ptr(), c->V, s0, s1); break;
    case PDF: import_kernel<PDF><<<grid, 256, 0, s>>>(c->g, lex, out.ptr(), c->V, s0, s1); break;
    case P32: import_kernel<P32><<<grid, 256, 0, s>>>(c->g, lex, out.ptr(), c->V, s0, s1); break;
    case P16: import_kernel<P16><<<grid, 256, 0, s>>>(c->g, lex, out.ptr(), c->V, s0, s1); break;
    case PB16: import_kernel<PB16><<<grid, 256, 0, s>>>(c->g, lex, out.ptr(), c->V, s0, s1); break;
    default: return QCD_ERR_ARG;
  }
  QCD_LAUNCHED();
  return QCD_OK;
}

static int export_range(qcd_ctx* c, const Rec& in, double* lex, int nrhs, long long s0, long long s1, cudaStream_t s) {
  if (in.nreal != 24) return QCD_ERR_ARG;
  if (s1 <= s0) return QCD_OK;
  dim3 grid((unsigned)((s1 - s0 + 255) / 256), nrhs);
  switch (in.prec) {
    case P64: export_kernel<P64><<<grid, 256, 0, s>>>(c->g, in.ptr(), lex, c->V, s0, s1); break;
    case PDF: export_kernel<PDF><<<grid, 256, 0, s>>>(c->g, in.ptr(), lex, c->V, s0, s1); break;
    case P32: export_kernel<P32><<<grid, 256, 0, s>>>(c->g, in.ptr(), lex, c->V, s0, s1); break;
    case P16: export_kernel<P16><<<grid, 256, 0, s>>>(c->g, in.ptr(), lex, c->V, s0, s1); break;
    case PB16: export_kernel<PB16><<<grid, 256, 0, s>>>(c->g, in.ptr(), lex, c->V, s0, s1); break;
    default: return QCD_ERR_ARG;
  }
  QCD_LAUNCHED();
  return QCD_OK;
}

int import_spinor(qcd_ctx* c, const double* lex, const Rec& out, int nrhs, cudaStream_t s) {
  return import_range(c, lex, out, nrhs, 0, c->V, s);
}

int export_spinor(qcd_ctx* c, const Rec& in, double* lex, int nrhs, cudaStream_t s) {
  return export_range(c, in, lex, nrhs, 0, c->V, s);
}

// Host transfers in slabs of time slices: with x0 the slowest lexicographic
// coordinate, the blocks of block time coordinates [n0, n1) are block indices
// [n0, n1) * bstr0 and lexicographic sites [n0, n1) * b0 * L1 L2 L3, so one
// slab is one contiguous range in both orders.  The copy of slab k+1 runs on
// the context's copy stream while slab k is imported (or exported) on s.
static int slabs(const qcd_ctx* c) {
  const int nb0 = c->g.nb[0];
  for (int k = 8; k > 1; --k)
    if (nb0 % k == 0) return k;
  return 1;
}

static int copy_stream(qcd_ctx* c, cudaStream_t* cs) {
  if (!c->copy_stream) QCD_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  *cs = c->copy_stream;
  return QCD_OK;
}

// one lattice's lexicographic host field -> stage (device) -> out (internal)
int upload_spinor(qcd_ctx* c, const double* host, double* stage, const Rec& out, cudaStream_t s) {
  cudaStream_t cs;
  QCD_TRY(copy_stream(c, &cs));
  const int n = slabs(c);
  const long long vs = c->V / n;  // sites per slab, both orders
  cudaEvent_t e;
  QCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEventRecord(e, s);  // the copies follow s's earlier work on the stage
  cudaStreamWaitEvent(cs, e, 0);
  cudaEventDestroy(e);
  for (int k = 0; k < n; ++k) {
    QCD_CUDA(cudaMemcpyAsync(stage + k * vs * 24, host + k * vs * 24, (size_t)vs * 24 * sizeof(double),
                             cudaMemcpyHostToDevice, cs));
    QCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEventRecord(e, cs);
    cudaStreamWaitEvent(s, e, 0);
    cudaEventDestroy(e);
    QCD_TRY(import_range(c, stage, out, 1, k * vs, (k + 1) * vs, s));
  }
  return QCD_OK;
}

int deliver_solution(Problem& p, cudaStream_t s) {
  qcd_ctx* c = p.c;
  if (!c->deliver_stream) {
    // the highest priority: its export CTAs take SM slots as the residual's free up,
    // so the copies start while the residual is still running
    int least = 0, greatest = 0;
    QCD_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    QCD_CUDA(cudaStreamCreateWithPriority(&c->deliver_stream, cudaStreamNonBlocking, greatest));
  }
  if (!p.dlv_event) QCD_CUDA(cudaEventCreateWithFlags(&p.dlv_event, cudaEventDisableTiming));
  cudaStream_t ds = c->deliver_stream;
  cudaEvent_t e;
  QCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEventRecord(e, s);  // after the update of x
  cudaStreamWaitEvent(ds, e, 0);
  cudaEventDestroy(e);
  if (p.dlv_stage)
    QCD_TRY(download_spinor(c, p.x, p.dlv_stage, p.dlv_lex, ds));
  else
    QCD_TRY(export_spinor(c, p.x, p.dlv_lex, 1, ds));
  QCD_CUDA(cudaEventRecord(p.dlv_event, ds));
  p.delivered = true;
  return QCD_OK;
}

// in (internal) -> stage -> the lexicographic host field; s waits for the copies
int download_spinor(qcd_ctx* c, const Rec& in, double* stage, double* host, cudaStream_t s) {
  cudaStream_t cs;
  QCD_TRY(copy_stream(c, &cs));
  const int n = slabs(c);
  const long long vs = c->V / n;
  cudaEvent_t e;
  for (int k = 0; k < n; ++k) {
    QCD_TRY(export_range(c, in, stage, 1, k * vs, (k + 1) * vs, s));
    QCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEventRecord(e, s);
    cudaStreamWaitEvent(cs, e, 0);
    cudaEventDestroy(e);
    QCD_CUDA(cudaMemcpyAsync(host + k * vs * 24, stage + k * vs * 24, (size_t)vs * 24 * sizeof(double),
                             cudaMemcpyDeviceToHost, cs));
  }
  QCD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEventRecord(e, cs);
  cudaStreamWaitEvent(s, e, 0);
  cudaEventDestroy(e);
  return QCD_OK;
}

// ------------------------------------------------------------------------
// gauge field
// ------------------------------------------------------------------------

// lexicographic (V, 4, 3, 3) complex128 -> internal FP64 full links;
// records max(|U U^+ - 1|, |det U - 1|) in *dev (as float bits, atomicMax)
__global__ void gauge_import_kernel(Geom g, const double* __restrict__ lex, double2* __restrict__ U64,
                                    unsigned int* dev) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  int x[4];
  global_coords(g, blk, r, x);
  const double2* src = (const double2*)lex + lex_index(g, x) * 36;
  float worst = 0.f;
  for (int mu = 0; mu < 4; ++mu) {
    cpx<double> u[3][3];
    for (int k = 0; k < 9; ++k) {
      double2 d = __ldg(src + mu * 9 + k);
      u[k / 3][k % 3] = {d.x, d.y};
      U64[((long long)(blk * 4 + mu) * 9 + k) * g.Vb + r] = d;
    }
    double dev_u = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        cpx<double> v = {0, 0};
        for (int k = 0; k < 3; ++k) v = cmadd(u[a][k], conjg(u[b][k]), v);
        double re = v.re - (a == b ? 1.0 : 0.0);
        dev_u = fmax(dev_u, fabs(re) + fabs(v.im));
      }
    cpx<double> det = cmul(u[0][0], cmul(u[1][1], u[2][2]) - cmul(u[1][2], u[2][1])) -
                      cmul(u[0][1], cmul(u[1][0], u[2][2]) - cmul(u[1][2], u[2][0])) +
                      cmul(u[0][2], cmul(u[1][0], u[2][1]) - cmul(u[1][1], u[2][0]));
    dev_u = fmax(dev_u, fabs(det.re - 1.0) + fabs(det.im));
    if (!(dev_u == dev_u)) dev_u = 1e30;  // NaN
    worst = fmaxf(worst, (float)fmin(dev_u, 1e30));
  }
  atomicMax(dev, __float_as_uint(worst));
}

int load_gauge_device(qcd_ctx* c, const double* lex_dev, cudaStream_t s) {
  ++c->gen;  // the links change (and their reduced-precision copies are freed)
  if (!c->U[P64]) {
    c->U_bytes[P64] = (size_t)c->V * GaugeLayout<P64>::bytes_per_site;
    if (cudaMalloc(&c->U[P64], c->U_bytes[P64]) != cudaSuccess) {
      c->U[P64] = nullptr;
      return QCD_ERR_NOMEM;
    }
  }
  for (int p = 1; p < 5; ++p)
    if (c->U[p]) {
      cudaFree(c->U[p]);
      c->U[p] = nullptr;
    }
  unsigned int* d_dev = (unsigned int*)c->d_scalars;
  QCD_CUDA(cudaMemsetAsync(d_dev, 0, sizeof(unsigned int), s));
  gauge_import_kernel<<<(unsigned)((c->V + 255) / 256), 256, 0, s>>>(c->g, lex_dev, (double2*)c->U[P64], d_dev);
  QCD_LAUNCHED();
  unsigned int h = 0;
  QCD_CUDA(cudaMemcpyAsync(&h, d_dev, sizeof(h), cudaMemcpyDeviceToHost, s));
  QCD_CUDA(cudaStreamSynchronize(s));
  float worst;
  memcpy(&worst, &h, sizeof(worst));
  c->gauge_loaded = true;
  c->clover_built = false;
  if (!(worst <= 1e-10f)) return QCD_ERR_NOT_SU3;
  return QCD_OK;
}

template <int P>
__global__ void gauge_compress_kernel(Geom g, const double2* __restrict__ U64, void* out) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int blk = (int)(s / g.Vb), r = (int)(s - (long long)blk * g.Vb);
  for (int mu = 0; mu < 4; ++mu) {
    float f[12];
    for (int k = 0; k < 6; ++k) {
      double2 d = U64[((long long)(blk * 4 + mu) * 9 + k) * g.Vb + r];
      f[2 * k] = (float)d.x;
      f[2 * k + 1] = (float)d.y;
    }
    if constexpr (P == P32) {
      float4* d = (float4*)out + ((long long)(blk * 4 + mu) * 3) * g.Vb + r;
      for (int k = 0; k < 3; ++k)
        d[(long long)k * g.Vb] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    } else {
      typedef typename Storage<P>::real hr;
      char* base = (char*)out + (long long)blk * g.Vb * 96;
      uint4 a;
      uint2 b;
      hr* ha = reinterpret_cast<hr*>(&a);
      hr* hb = reinterpret_cast<hr*>(&b);
      for (int e = 0; e < 8; ++e) ha[e] = from_f<P>(f[e]);
      for (int e = 0; e < 4; ++e) hb[e] = from_f<P>(f[8 + e]);
      ((uint4*)base)[(long long)mu * g.Vb + r] = a;
      ((uint2*)(base + (long long)64 * g.Vb))[(long long)mu * g.Vb + r] = b;
    }
  }
}

// FP64 links -> double-float pairs (element by element, same layout)
__global__ void gauge_split_kernel(const double2* __restrict__ in, float4* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = in[i];
  const df a = df_from_f64(v.x), b = df_from_f64(v.y);
  out[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
}

int ensure_gauge(qcd_ctx* c, int prec, cudaStream_t s) {
  if (!c->gauge_loaded) return QCD_ERR_STATE;
  if (c->U[prec]) return QCD_OK;
  ++c->gen;
  size_t bytes = (size_t)c->V * ((prec == P64 || prec == PDF) ? GaugeLayout<P64>::bytes_per_site
                                 : (prec == P32 ? GaugeLayout<P32>::bytes_per_site
                                                : GaugeLayout<P16>::bytes_per_site));
  if (cudaMalloc(&c->U[prec], bytes) != cudaSuccess) {
    c->U[prec] = nullptr;
    return QCD_ERR_NOMEM;
  }
  c->U_bytes[prec] = bytes;
  unsigned grid = (unsigned)((c->V + 255) / 256);
  const double2* U64 = (const double2*)c->U[P64];
  switch (prec) {
    case P32: gauge_compress_kernel<P32><<<grid, 256, 0, s>>>(c->g, U64, c->U[prec]); break;
    case P16: gauge_compress_kernel<P16><<<grid, 256, 0, s>>>(c->g, U64, c->U[prec]); break;
    case PB16: gauge_compress_kernel<PB16><<<grid, 256, 0, s>>>(c->g, U64, c->U[prec]); break;
    case PDF: {  // all 18 reals of every link as double-float pairs, FP64 order
      const long long n = c->V * 4 * 9;
      gauge_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(U64, (float4*)c->U[prec], n);
      break;
    }
    default: return QCD_ERR_ARG;
  }
  QCD_LAUNCHED();
  return QCD_OK;
}

// ------------------------------------------------------------------------
// record conversion between precisions (spinors: 24 reals, clover: 72)
// ------------------------------------------------------------------------
template <int PI, int PO, int N>
__global__ void convert_kernel(int Vb, long long V, FieldPtr in, FieldPtr out) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int blk = (int)(s / Vb), r = (int)(s - (long long)blk * Vb);
  if constexpr (PI == P64 && (PO == P64 || PO == PDF)) {
    double v[N];
    load_record<PI, N, double>(in, Vb, blk, r, v);
    store_record<PO, N, double>(out, Vb, blk, r, v);
  } else if constexpr (PI == P64) {
    double v[N];
    load_record<PI, N, double>(in, Vb, blk, r, v);
    float w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = (float)v[k];
    store_record<PO, N, float>(out, Vb, blk, r, w);
  } else if constexpr (PO == P64) {
    float w[N];
    load_record<PI, N, float>(in, Vb, blk, r, w);
    double v[N];
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = w[k];
    store_record<PO, N, double>(out, Vb, blk, r, v);
  } else {
    float w[N];
    load_record<PI, N, float>(in, Vb, blk, r, w);
    store_record<PO, N, float>(out, Vb, blk, r, w);
  }
}

template <int N>
static int convert_n(qcd_ctx* c, const Rec& in, const Rec& out, cudaStream_t s) {
  unsigned grid = (unsigned)((c->V + 255) / 256);
  int Vb = c->g.Vb;
  long long V = c->V;
#define CV(PI, PO)                                                                     \
  if (in.prec == PI && out.prec == PO) {                                               \
    convert_kernel<PI, PO, N><<<grid, 256, 0, s>>>(Vb, V, in.ptr(), out.ptr());        \
    QCD_LAUNCHED();                                                      \
    return QCD_OK;                                                                     \
  }
  CV(P64, P64) CV(P64, P32) CV(P64, P16) CV(P64, PB16) CV(P64, PDF)
  CV(P32, P64) CV(P32, P32) CV(P32, P16) CV(P32, PB16)
  CV(P16, P64) CV(P16, P32) CV(PB16, P64) CV(PB16, P32)
#undef CV
  return QCD_ERR_UNSUPPORTED;
}

int convert_rec(qcd_ctx* c, const Rec& in, const Rec& out, cudaStream_t s) {
  if (in.nreal != out.nreal) return QCD_ERR_ARG;
  if (in.nreal == 24) return convert_n<24>(c, in, out, s);
  if (in.nreal == 72) return convert_n<72>(c, in, out, s);
  return QCD_ERR_ARG;
}

// element by element: out32 = f64_to_f32(in64), out64 = f32_to_f64(in32), the
// integer-pipe conversions of the SAP edges and the refinement kernels
__global__ void convert_check_kernel(const double* __restrict__ in64, const float* __restrict__ in32,
                                     float* __restrict__ out32, double* __restrict__ out64, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    out32[i] = f64_to_f32(in64[i]);
    out64[i] = f32_to_f64(in32[i]);
  }
}

int convert_check(const double* in64, const float* in32, float* out32, double* out64, long long n, cudaStream_t s) {
  if (n == 0) return QCD_OK;
  const long long blocks = (n + 255) / 256;
  convert_check_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(in64, in32, out32, out64, n);
  QCD_LAUNCHED();
  return QCD_OK;
}

}  // namespace qcd
