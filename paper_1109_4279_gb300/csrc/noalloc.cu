// qcd_apply_D_noalloc: the FP64 operator apply of qcd_apply_D without any
// device allocation.
//
// qcd_apply_D stages the caller's lexicographic spinor into the block-major
// even/odd layout and back through two temporary fields that it allocates and
// frees on every call.  Some callers cannot have a library do that: programs
// that hand all device memory to their own pool allocator with a fixed budget
// (a cudaMalloc behind its back can fail or fragment the pool), and
// latency-sensitive loops in which cudaFree's implicit device-wide
// synchronisation would stall every other stream.  This variant keeps the two
// staging fields in one file-scope device array instead.
//
// Limits and sharing rules:
//  * at most kMaxSites = 65536 lattice sites (e.g. 16^4); larger lattices get
//    QCD_ERR_TOO_LARGE;
//  * the array (24 MiB) exists on every GPU that loads the library, until the
//    process exits;
//  * all calls share it and it keeps the last call's contents: every element
//    a call reads is first written by the same call (the whole input field is
//    converted, the whole output field is computed), so nothing needs
//    clearing;
//  * calls that overlap on the GPU (different streams, or different contexts
//    on the same device, without ordering between them) race on the array;
//  * the first call on each device looks up the array's device address with
//    cudaGetSymbolAddress; make that first call before any stream capture;
//  * the looked-up address is kept for the life of the process: after
//    cudaDeviceReset (which destroys the context the address belongs to) this
//    entry point must not be called again in the same process;
//  * kernel profiling (qcd_profile_enable) records CUDA events, which are
//    created on demand: a context with profiling on gets QCD_ERR_STATE.
#include <mutex>

#include "internal.h"

namespace qcd {

static constexpr long long kMaxSites = 65536;
// two FP64 spinor fields in internal layout: 12 double2 per site each
static __device__ __align__(256) double2 g_noalloc_scratch[2 * 12 * kMaxSites];

static constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (looked up once per device)
static int scratch_address(void** out) {
  int dev = 0;
  QCD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return QCD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return QCD_OK;
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_apply_D_noalloc(qcd_ctx* c, const double* in, double* out, int dagger, void* stream) {
  if (!c || !in || !out) return QCD_ERR_ARG;
  if (c->V > kMaxSites) return QCD_ERR_TOO_LARGE;
  if (!c->clover_built || !c->U[P64] || !c->A[P64].data || c->prof) return QCD_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  QCD_TRY(scratch_address(&base));
  Rec a, b;  // views of the static array; never passed to rec_free
  a.prec = b.prec = P64;
  a.nreal = b.nreal = 24;
  a.data = base;
  b.data = (char*)base + (size_t)c->V * 12 * sizeof(double2);
  QCD_TRY(import_spinor(c, in, a, 1, s));
  QCD_TRY(dirac_apply(c, a, b, dagger, s));
  return export_spinor(c, b, out, 1, s);
}
