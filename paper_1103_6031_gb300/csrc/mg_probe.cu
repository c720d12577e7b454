// Issue rate of the FP64 pipe, measured on the device in use.
//
// The float64 stencil kernels of this library need more FP64 instructions per
// HBM byte than the GPU's FP64 pipe can issue at its copy bandwidth, so their
// roofline is the FP64 issue rate, not HBM.  This probe measures that rate the
// way the stencils use the pipe: every thread runs 8 independent chains of
// fused multiply-adds (enough independent work per warp to cover the pipe's
// latency), on a grid of 8 blocks of 256 threads per SM, timed with CUDA events.
//
// The event-pair floor: what a CUDA-event pair around one kernel node of a CUDA graph
// reads for a kernel that does nothing, the fixed cost inside every event-timed launch
// of the profiled kernel families.
#include <cuda_runtime.h>

#include <vector>

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

__global__ void k_nothing() {}

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

extern "C" mg_status mg_event_pair_floor(int pairs, void* cuda_stream, double* us) {
  if (!us || pairs < 1 || pairs > 1024) return MG_EINVAL;
  *us = 0.0;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::vector<cudaEvent_t> ev(2 * pairs, nullptr);
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t joined = nullptr;
  mg_status st = MG_OK;
  for (cudaEvent_t& e : ev)
    if (st == MG_OK && cudaEventCreate(&e) != cudaSuccess) st = MG_ECUDA;
  if (st == MG_OK && (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&joined, cudaEventDisableTiming) != cudaSuccess))
    st = MG_ECUDA;
  // the same form as a profiled launch: event record node, kernel node, event record node
  if (st == MG_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    st = MG_ECUDA;
  if (st == MG_OK) {
    bool ok = true;
    for (int i = 0; i < pairs && ok; ++i) {
      ok = cudaEventRecordWithFlags(ev[2 * i], cs, cudaEventRecordExternal) == cudaSuccess;
      k_nothing<<<1, 32, 0, cs>>>();
      ok = ok && cudaGetLastError() == cudaSuccess &&
           cudaEventRecordWithFlags(ev[2 * i + 1], cs, cudaEventRecordExternal) == cudaSuccess;
    }
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (!ok || e != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = MG_ECUDA;
  }
  // ordered after the caller's stream; the first replay warms the graph up
  if (st == MG_OK && (cudaEventRecord(joined, s) != cudaSuccess ||
                      cudaStreamWaitEvent(cs, joined, 0) != cudaSuccess ||
                      cudaGraphLaunch(ge, cs) != cudaSuccess || cudaGraphLaunch(ge, cs) != cudaSuccess ||
                      cudaStreamSynchronize(cs) != cudaSuccess))
    st = MG_ECUDA;
  double sum = 0.0;
  for (int i = 0; i < pairs && st == MG_OK; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) st = MG_ECUDA;
    sum += ms;
  }
  if (st == MG_OK) *us = 1e3 * sum / pairs;
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (joined) cudaEventDestroy(joined);
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return st;
}
