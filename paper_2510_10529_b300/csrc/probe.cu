// Arithmetic-rate probes of this device: FP64 FMA, FP32 FMA (scalar and
// packed pairs) and the TF32 tensor pipe.  They give the roofline
// denominators of kernels bound by arithmetic rather than by memory.  Each
// probe fills the GPU with independent FMA chains on register operands (or
// tensor-core MMA chains on shared-memory operands), with no memory traffic,
// and is timed with CUDA events at the clocks the GPU runs at.
#include "internal.h"

namespace invdft {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;      // independent accumulators per thread

__global__ void __launch_bounds__(kProbeThreads) fma64_probe(int iters, double seed, double *out) {
  double a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = seed + threadIdx.x * 1e-3 + k;
  const double b = 0.9999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == 12345.678) out[blockIdx.x] = s;       // keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) fma32_probe(int iters, float seed, float *out) {
  float a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = seed + threadIdx.x * 1e-3f + k;
  const float b = 0.9999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == 12345.678f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) ffma2_probe(int iters, float seed, float *out) {
  float2 a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = make_float2(seed + k, seed - k + threadIdx.x * 1e-3f);
  const float2 b = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k].x + a[k].y;
  if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace invdft

using namespace invdft;

extern "C" invdft_status invdft_peak_probe(int kind, double *tflops, double *ms_out, void *stream) {
  if (!tflops || kind < 0 || kind > 3) {
    set_global_error("peak_probe: kind must be 0 (FP64 FMA), 1 (FP32 FMA), 2 (packed FP32 "
                     "FMA) or 3 (TF32 tensor cores)");
    return INVDFT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  double *scratch = nullptr;
  int *err = nullptr;
  if (cudaMalloc(&scratch, 4096 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaMemset(err, 0, sizeof(int)) != cudaSuccess) {
    if (scratch) cudaFree(scratch);
    set_global_error("peak_probe: scratch allocation failed");
    return INVDFT_ECUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = nsm * 8;
  double flops = 0.0;
  float ms = 0.f;
  cudaError_t rc = cudaSuccess;
  for (int rep = 0; rep < 2 && rc == cudaSuccess; ++rep) {    // the first run warms up
    cudaEventRecord(e0, s);
    if (kind == 0) {
      const int iters = 4096;
      ::invdft::count_launch();
      fma64_probe<<<grid, kProbeThreads, 0, s>>>(iters, 1.0, scratch);
      flops = 2.0 * grid * kProbeThreads * iters * kProbeChains;
    } else if (kind == 1) {
      const int iters = 1 << 16;
      ::invdft::count_launch();
      fma32_probe<<<grid, kProbeThreads, 0, s>>>(iters, 1.f, (float *)scratch);
      flops = 2.0 * grid * kProbeThreads * iters * kProbeChains;
    } else if (kind == 2) {
      const int iters = 1 << 15;
      ::invdft::count_launch();
      ffma2_probe<<<grid, kProbeThreads, 0, s>>>(iters, 1.f, (float *)scratch);
      flops = 4.0 * grid * kProbeThreads * iters * kProbeChains;
    } else {
      rc = launch_tf32_probe(2 * nsm, 4000, err, &flops, s);
    }
    if (rc == cudaSuccess) rc = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (rc == cudaSuccess) rc = cudaEventSynchronize(e1);
  }
  int herr = 0;
  if (rc == cudaSuccess) rc = cudaEventElapsedTime(&ms, e0, e1);
  if (rc == cudaSuccess) rc = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  cudaFree(err);
  if (rc != cudaSuccess) {
    set_global_error(cudaGetErrorString(rc));
    return INVDFT_ECUDA;
  }
  if (herr) {
    set_global_error("peak_probe: the tensor-core probe's wait gave up");
    return INVDFT_ETIMEOUT;
  }
  *tflops = flops / ((double)ms * 1e9);
  if (ms_out) *ms_out = ms;
  return INVDFT_OK;
}
