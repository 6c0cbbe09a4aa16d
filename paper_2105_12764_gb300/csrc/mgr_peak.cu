// mgr_peak.cu -- measured FP64 fused multiply-add throughput of a device.
//
// The plain FP64 form of the level pass is bound by the FP64 pipe, not by
// HBM, so its roofline denominator is the rate at which the SMs retire FP64
// FMAs.  This measures it the way the pass would see it: every thread runs
// eight independent FMA chains (enough independent work to keep the pipe
// full), over a grid of four 256-thread CTAs per SM, timed with CUDA events
// after a warm-up launch; the best of three launches is reported.
#include <cuda_runtime.h>

#include <algorithm>

#include "mgr_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_dfma_rate(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" int mgr_fp64_fma_rate(int device, double* fma_per_second) {
  if (!fma_per_second) return MGR_EINVAL;
  *fma_per_second = 0.0;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  if (device < 0 || device >= n) return MGR_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * kCtasPerSm;
  const int iters = 8192;  // about 10 ms on a GB300 at its nominal FP64 rate
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  int rc = MGR_OK;
  if (cudaMalloc(&out, sizeof(double) * size_t(blocks) * kThreads) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    rc = MGR_ECUDA;
  }
  double best = 0.0;
  for (int rep = 0; rc == MGR_OK && rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    k_dfma_rate<<<blocks, kThreads, 0, st>>>(out, iters, 0.999999999, 1e-9);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = MGR_ECUDA;
      break;
    }
    const double fmas = double(blocks) * kThreads * kChains * iters;
    if (rep > 0 && ms > 0.f) best = std::max(best, fmas / (double(ms) * 1e-3));  // rep 0 warms up
  }
  if (st) cudaStreamDestroy(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaGetLastError();
  cudaSetDevice(prev);
  if (rc == MGR_OK) *fma_per_second = best;
  return rc;
}
