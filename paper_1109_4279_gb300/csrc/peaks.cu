// Arithmetic peaks of the GPU the library runs on, measured: the denominators
// of the ALU rooflines of the block solver (FP32) and of the FP64 recursion.
//
// Each kernel keeps eight independent fused multiply-add chains per thread in
// registers (no memory traffic inside the timed loop) on a grid of several
// CTAs per SM, long enough (tens of milliseconds) for the clock to settle.
// Three forms: scalar FP32 FMA, packed FP32x2 FMA (the instruction the
// operator and block-solver kernels use for SU(3) products), and FP64 FMA.
// Throughput counts 2 flops per lane per multiply-add.
#include "internal.h"

namespace qcd {

static constexpr int kPeakThreads = 256;
static constexpr int kPeakChains = 8;

template <typename T>
__device__ __forceinline__ T fma_step(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_step<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_step<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float2 fma_step<float2>(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T peak_seed(float v);
template <>
__device__ __forceinline__ float peak_seed<float>(float v) { return v; }
template <>
__device__ __forceinline__ double peak_seed<double>(float v) { return (double)v; }
template <>
__device__ __forceinline__ float2 peak_seed<float2>(float v) { return make_float2(v, v + 0.5f); }

__device__ __forceinline__ float peak_sum(float v) { return v; }
__device__ __forceinline__ float peak_sum(double v) { return (float)v; }
__device__ __forceinline__ float peak_sum(float2 v) { return v.x + v.y; }

// iters rounds of kPeakChains dependent-per-chain multiply-adds; the result is
// stored only if it is exactly a value the chains cannot reach, so nothing is
// written in practice but the work cannot be removed
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, float a, float b, float* sink) {
  T acc[kPeakChains];
  const T ma = peak_seed<T>(a), mb = peak_seed<T>(b);
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) acc[j] = peak_seed<T>(threadIdx.x * 1e-3f + j);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kPeakChains; ++j) acc[j] = fma_step<T>(acc[j], ma, mb);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += peak_sum(acc[j]);
  if (s == -12345.678f) sink[blockIdx.x] = s;
}

// TFLOP/s of one kernel form: reps launches of `iters` rounds each
template <typename T>
static int time_peak(int lanes_per_elem, int iters, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  QCD_CUDA(cudaGetDevice(&dev));
  QCD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * 8;
  float* sink = nullptr;
  QCD_CUDA(cudaMalloc(&sink, sizeof(float) * grid));
  // a and b keep the chains bounded: x -> 0.999 x + 1e-3 converges to 1
  fma_peak_kernel<T><<<grid, kPeakThreads, 0, s>>>(iters / 8, 0.999f, 1e-3f, sink);  // warm-up (clock ramp)
  QCD_LAUNCHED();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int reps = 3;
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) {
    fma_peak_kernel<T><<<grid, kPeakThreads, 0, s>>>(iters, 0.999f, 1e-3f, sink);
    QCD_LAUNCHED();
  }
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double fmas = (double)grid * kPeakThreads * iters * 16.0 * kPeakChains * lanes_per_elem * reps;
  *tflops = ms > 0 ? 2.0 * fmas / (ms * 1e-3) / 1e12 : 0.0;
  return QCD_OK;
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_measure_alu_peaks(double* fp32_tflops, double* fp32x2_tflops, double* fp64_tflops, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  double v = 0;
  if (fp32_tflops) {
    QCD_TRY(time_peak<float>(1, 4096, &v, s));
    *fp32_tflops = v;
  }
  if (fp32x2_tflops) {
    QCD_TRY(time_peak<float2>(2, 2048, &v, s));
    *fp32x2_tflops = v;
  }
  if (fp64_tflops) {
    QCD_TRY(time_peak<double>(1, 64, &v, s));
    *fp64_tflops = v;
  }
  return QCD_OK;
}
