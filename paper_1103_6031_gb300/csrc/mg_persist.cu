// The persistent batch kernel: the float32 V-cycles of many hierarchies in one launch
// over a work list of (hierarchy, level operation, block range) items.
//
// A block of 128 threads repeatedly takes the next item (one atomic counter), waits
// until its hierarchy has completed every earlier operation of its chain (a per-
// hierarchy counter read with acquire semantics; the wait is bounded by wait_ns of
// global time and polls the launch's error word), runs the item's blocks through the
// same bodies the stream kernels run (mg_vbody.cuh, with plain loads, since items read
// what earlier items of the launch wrote), and counts the item done; the block that
// completes an operation's last item publishes the hierarchy's counter with release
// semantics.  Items are handed out in chain order, so every item a block waits for
// was handed out earlier to a block that is running: with every block resident, the
// launch cannot deadlock; a wait that still runs out (a defect) sets the error word,
// and every block stops at its next wait or item.
#include <cstring>
#include <vector>

#include "mg_persist.h"
#include "mg_vbody.cuh"

namespace mgk {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

template <int ORDER>
__device__ __forceinline__ void run_block(const POp& op, const CfW<float>& w, int blk) {
  const int tid = threadIdx.x;
  switch (op.kind) {
    case P_ZERO: {
      const long long e0 = (long long)blk * kZeroPerBlock;
      const long long e1 = min(e0 + kZeroPerBlock, op.n);
      for (long long e = e0 + tid; e < e1; e += kPersistThreads) op.out0[e] = 0.f;
      break;
    }
    case P_SMOOTH: {
      const Blk b{blk % op.gx, (blk / op.gx) % op.gy, blk / (op.gx * op.gy), tid & 31, tid >> 5};
      smooth_half_body<ORDER, float, Weak>(op.F, op.in0, op.out0, op.in1, op.s[0], op.colour,
                                           op.periodic, kPersistThreads / kVPairX, b);
      break;
    }
    case P_CF_FLUX:
      cf_flux_body<ORDER, float>(op.F, op.out0, op.fs, w, op.in0, op.in1, op.s[0], op.s[1],
                                 op.s[2], op.s[3], op.s[4], 1,
                                 (long long)blk * kPersistThreads + tid);
      break;
    case P_GHOST_PERIODIC:
      ghost_periodic_body<float>(op.F, op.out0, (long long)blk * kPersistThreads + tid);
      break;
    case P_RESTRICT: {
      const Blk b{blk % op.gx, (blk / op.gx) % op.gy, blk / (op.gx * op.gy), tid & 31, tid >> 5};
      residual_restrict_body<ORDER, float, Weak>(op.F, op.in0, op.in1, op.s[0], op.P, op.out0,
                                                 op.out1, op.out2, op.off, op.cn, op.periodic, b);
      break;
    }
    case P_FAS: {
      const Blk b{blk % op.gx, (blk / op.gx) % op.gy, blk / (op.gx * op.gy), tid & 31, tid >> 5};
      fas_source_body<ORDER, float, Weak>(op.P, op.in0, op.out0, op.s[0], op.off, op.cn, b);
      break;
    }
    case P_COARSEST:
      coarsest_body<float, Weak>(op.F, op.in0, op.out0, op.kern, blk, tid);
      break;
    case P_TANG:
      cf_tangential_body<ORDER, float, Weak>(op.F, op.P, op.in0, op.off, op.fs, w, op.s[0],
                                             op.out0, op.out1,
                                             (long long)blk * kPersistThreads + tid);
      break;
    case P_PROLONG: {
      const Blk b{blk % op.gx, (blk / op.gx) % op.gy, blk / (op.gx * op.gy), tid & 31, tid >> 5};
      prolong_body<float, Weak>(op.F, op.out0, op.P, op.in0, op.in1, op.off, op.cn, op.periodic, b);
      break;
    }
    default:
      break;
  }
}

__global__ void __launch_bounds__(kPersistThreads)
    k_persist(const POp* __restrict__ ops, int nops, long long total,
              const CfW<float>* __restrict__ wts, PState* st, int* done, int* count,
              unsigned long long wait_ns) {
  __shared__ int s_op;
  __shared__ long long s_item;
  __shared__ int s_go;
  for (;;) {
    if (threadIdx.x == 0) {
      int go = 0, j = 0;
      const long long it = (long long)atomicAdd(&st->next, 1ULL);
      if (it < total && ld_volatile(&st->err) == 0u) {
        // the op whose items hold `it`: the last j with ops[j].tile0 <= it
        int lo = 0, hi = nops - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (ops[mid].tile0 <= it) lo = mid;
          else hi = mid - 1;
        }
        j = lo;
        const int m = ops[j].member, seq = ops[j].seq;
        go = 1;
        if (ld_acquire(done + m) < seq) {
          const unsigned long long t0 = global_ns();
          while (ld_acquire(done + m) < seq) {
            if (ld_volatile(&st->err) != 0u) {
              go = 0;
              break;
            }
            if (global_ns() - t0 > wait_ns) {
              atomicOr(&st->err, 1u);
              go = 0;
              break;
            }
            __nanosleep(128);
          }
        }
      }
      s_item = it;
      s_op = j;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const POp& op = ops[s_op];
    const CfW<float>& w = wts[op.member];
    const int lt = (int)(s_item - op.tile0);
    const int b0 = lt * op.per_tile;
    const int b1 = min(b0 + op.per_tile, op.nblk);
    for (int blk = b0; blk < b1; ++blk) {
      switch (op.order) {
        case 2: run_block<2>(op, w, blk); break;
        case 4: run_block<4>(op, w, blk); break;
        default: run_block<6>(op, w, blk); break;
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const int c = atomicAdd(count + s_op, 1) + 1;
      if (c == op.ntiles) st_release(done + op.member, op.seq + 1);
    }
  }
}

__global__ void k_persist_flags(const PState* __restrict__ st, unsigned* const* __restrict__ flags,
                                int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flags[i] && st->err) atomicOr(flags[i], 1u);
}

}  // namespace

cudaError_t launch_persist_flags(const PState* st, unsigned* const* flags, int n, cudaStream_t s) {
  if (n < 1) return cudaErrorInvalidValue;
  k_persist_flags<<<(n + 127) / 128, 128, 0, s>>>(st, flags, n);
  return cudaGetLastError();
}

cudaError_t launch_persist(const POp* ops, int nops, long long total, const void* wts,
                           PState* st, int* done, int* count, unsigned long long wait_ns,
                           int grid, cudaStream_t s) {
  if (nops < 1 || total < 1 || grid < 1) return cudaErrorInvalidValue;
  k_persist<<<grid, kPersistThreads, 0, s>>>(ops, nops, total,
                                             static_cast<const CfW<float>*>(wts), st, done,
                                             count, wait_ns);
  return cudaGetLastError();
}

cudaError_t persist_grid(int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kPersistThreads, 0);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) *grid = sms * per_sm;
  return e;
}

size_t persist_weight_bytes() { return sizeof(CfW<float>); }

void persist_weights(const CfWeights& w, void* dst) {
  const CfW<float> o = cf_weights_as<float>(w);
  std::memcpy(dst, &o, sizeof(o));
}

}  // namespace mgk

// Self-test of the bounded dependency wait (no counterpart in the paper): a work list
// whose second item depends on an operation that does not exist, so its wait can never
// be satisfied; with a 100 ms limit the block gives up, sets the error word and the
// launch ends.
extern "C" mg_status mg_selftest_persist_wait(void) {
  using namespace mgk;
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };  // every region 256-aligned
  const size_t off_w = up(2 * sizeof(POp));
  const size_t off_z = up(off_w + persist_weight_bytes());
  const size_t off_s = up(off_z + 1024 * sizeof(float));
  const size_t off_d = up(off_s + sizeof(PState));
  const size_t bytes = off_d + 4 * sizeof(int);
  char* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) return MG_ENOMEM;
  POp ops[2];
  std::memset(ops, 0, sizeof(ops));
  for (int q = 0; q < 2; ++q) {
    ops[q].kind = P_ZERO;
    ops[q].order = 2;
    ops[q].member = 0;
    ops[q].seq = q == 0 ? 0 : 2;  // seq 1 does not exist: the second wait never ends
    ops[q].nblk = 1;
    ops[q].per_tile = 1;
    ops[q].ntiles = 1;
    ops[q].tile0 = q;
    ops[q].out0 = reinterpret_cast<float*>(d + off_z);
    ops[q].n = 1024;
  }
  std::vector<unsigned char> w(persist_weight_bytes(), 0);
  PState* st = reinterpret_cast<PState*>(d + off_s);
  int* done = reinterpret_cast<int*>(d + off_d);  // done[1] (one member), then count[2]
  int* count = done + 2;
  cudaStream_t s = nullptr;
  mg_status r = MG_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMemcpyAsync(d, ops, sizeof(ops), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d + off_w, w.data(), w.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(d + off_s, 0, bytes - off_s, s) != cudaSuccess ||
      launch_persist(reinterpret_cast<const POp*>(d), 2, 2, d + off_w, st, done, count,
                     100000000ull, 2, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    r = MG_ECUDA;
  } else {
    unsigned err = 0;
    if (cudaMemcpy(&err, &st->err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) r = MG_ECUDA;
    else r = err ? MG_ETIMEOUT : MG_OK;
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(d);
  return r;
}
