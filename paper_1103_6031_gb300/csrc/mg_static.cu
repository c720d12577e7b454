// 2LPT source on one periodic level with no device allocation.
//
// Some callers cannot allocate device memory when they need this result: a
// host application whose device memory is entirely reserved by its own pool
// allocator, a plugin that is handed a stream but no allocator, or code that
// must not risk the implicit device synchronisation of cudaMalloc/cudaFree.
// This entry point serves them: its working memory (a ghost-padded copy of
// phi, a padded tau and three padded first-derivative arrays) lives in one
// file-scope __device__ array that every
// GPU holds from module load until process exit, so the call itself makes no
// allocation.  The caller passes only the input phi and the output tau.
//
// The device address of the array is looked up once per device, on the first
// call made while that device is current (cudaGetSymbolAddress); make that
// first call outside any stream capture.  The address is kept until the process
// exits: after cudaDeviceReset the module is loaded again, possibly elsewhere, so
// this entry point must not be called on a device that was reset in the same
// process.  All calls share the array and each
// call overwrites every element it later reads, so nothing carries over from
// a previous call; two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "mg.h"
#include "mg_internal.h"

namespace {

// Capacity of the static working array: five padded float64 grids.
constexpr long long kStaticElems = (16LL << 20) / 8;  // 16 MiB
static __device__ __align__(256) double g_static_work[kStaticElems];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_addr[kMaxDevices] = {nullptr};

void put_msg(char* err, size_t len, const char* text) {
  if (err && len) snprintf(err, len, "%s", text);
}

}  // namespace

extern "C" mg_status mg_lpt2_source_periodic_static(const double* phi, double* tau, int n0,
                                                    int n1, int n2, double box, int order,
                                                    void* cuda_stream, char* err, size_t len) {
  put_msg(err, len, "");
  if (!phi || !tau) {
    put_msg(err, len, "phi and tau must be device pointers");
    return MG_EINVAL;
  }
  if (order != 2 && order != 4 && order != 6) {
    put_msg(err, len, "order must be 2, 4 or 6");
    return MG_EINVAL;
  }
  const int g = order / 2;
  if (n0 < g || n1 < g || n2 < g || n0 < 2 || n1 < 2 || n2 < 2 || !(box > 0.0)) {
    put_msg(err, len, "every side must be >= max(2, order/2) and box > 0");
    return MG_EINVAL;
  }
  const mgk::Grid G = mgk::make_grid(n0, n1, n2, g);
  const long long need = 5 * mgk::grid_elems(G);
  if (need > kStaticElems) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "grid %dx%dx%d needs %lld float64 of working memory; the static array holds %lld "
             "(about 64^3 cells at order 6)", n0, n1, n2, need, kStaticElems);
    put_msg(err, len, buf);
    return MG_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    put_msg(err, len, "no usable current CUDA device");
    return MG_ECUDA;
  }
  double* work = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_static_work);
      if (e != cudaSuccess || !p) {
        put_msg(err, len, cudaGetErrorString(e));
        return MG_ECUDA;
      }
      g_addr[dev] = static_cast<double*>(p);
    }
    work = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* phi_pad = work;
  double* tau_pad = work + mgk::grid_elems(G);
  const double h = box / n0;
  cudaError_t e = mgk::launch_pack(G, phi, phi_pad, 0.0, s);
  if (e == cudaSuccess) e = mgk::launch_ghost_periodic<double>(G, phi_pad, s);
  if (e == cudaSuccess)
    e = mgk::launch_lpt2_source(order, G, phi_pad, 1.0 / (h * h), tau_pad,
                                work + 2 * mgk::grid_elems(G), s);
  if (e == cudaSuccess) e = mgk::launch_unpack(G, tau_pad, tau, s);
  if (e != cudaSuccess) {
    put_msg(err, len, cudaGetErrorString(e));
    return MG_ECUDA;
  }
  return MG_OK;
}
