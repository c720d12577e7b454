// Issue rate of the FP64 pipe, measured on the device in use.
//
// The float64 stencil kernels of this library need more FP64 instructions per
// HBM byte than the GPU's FP64 pipe can issue at its copy bandwidth, so their
// roofline is the FP64 issue rate, not HBM.  This probe measures that rate the
// way the stencils use the pipe: every thread runs 8 independent chains of
// fused multiply-adds (enough independent work per warp to cover the pipe's
// latency), on a grid of 8 blocks of 256 threads per SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "mg.h"

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kBlock) k_dfma_chains(int iters, double a, double b,
                                                         double* __restrict__ sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // never true for the arguments the host passes; keeps the chains live
  if (s == 1234.5) sink[blockIdx.x * kBlock + threadIdx.x] = s;
}

}  // namespace

extern "C" mg_status mg_fp64_fma_rate(int iters, void* cuda_stream, double* fma_per_s) {
  if (!fma_per_s || iters < 16 || iters > (1 << 22)) return MG_EINVAL;
  *fma_per_s = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return MG_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int blocks = sms * kBlocksPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mg_status st = MG_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = MG_ECUDA;
  // a = 1 - 2^-40, b = 2^-50: every chain stays near its start value, far from 1234.5
  const double a = 1.0 - 9.094947017729282e-13, b = 8.881784197001252e-16;
  if (st == MG_OK) {
    k_dfma_chains<<<blocks, kBlock, 0, s>>>(iters / 8, a, b, nullptr);  // warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) st = MG_ECUDA;
  }
  if (st == MG_OK) {
    k_dfma_chains<<<blocks, kBlock, 0, s>>>(iters, a, b, nullptr);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess)
      st = MG_ECUDA;
  }
  float ms = 0.f;
  if (st == MG_OK && (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)))
    st = MG_ECUDA;
  if (st == MG_OK)
    *fma_per_s = (double)blocks * kBlock * kChains * (double)iters / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}
