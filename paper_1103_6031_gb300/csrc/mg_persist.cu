// The persistent batch kernel: the float32 V-cycles of many hierarchies in one launch
// over a work list of (hierarchy, level operation, block range) items.
//
// Each hierarchy's operations form a chain (ops[mop0[m] .. mop0[m] + mops[m]), items
// numbered along the chain); only the first incomplete operation of a chain is open.
// A block of 128 threads scans the hierarchies (from a rotating start) for one whose
// open operation still has items, takes one, runs the item's blocks through the same bodies the stream kernels run
// (mg_vbody.cuh, with plain loads, since items read what earlier items of the launch
// wrote), and counts it done; the block that completes an operation's last item opens
// the next one by publishing the chain's done counter with release semantics (a taker
// orders its item after that release with an acquire fence).  Items are tickets from
// the operation's own counter, so a ticket drawn late (past the operation's items) is
// dropped without retries.  A block never waits on an item it holds, so every
// taken item completes; a block that finds nothing open waits, and a wait longer than
// wait_ns without a single item (a defect: no chain can advance) sets the error word,
// after which every block stops.
#include <cstring>
#include <vector>

#include "mg_persist.h"
#include "mg_vbody.cuh"

namespace mgk {

namespace {

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acquire() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
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

// At least 8 blocks per SM (64 registers): the stencil bodies are latency-bound on L1
// and need the warps; at 96 registers 5 blocks fit.
__global__ void __launch_bounds__(kPersistThreads, 8)
    k_persist(const POp* __restrict__ ops, const int* __restrict__ mop0, const int* __restrict__ mops,
              int members, int active, const CfW<float>* __restrict__ wts, PState* st, int* done,
              int* taken, int* count, unsigned long long wait_ns) {
  __shared__ int s_op, s_lt, s_go;
  unsigned long long idle_since = 0;
  unsigned backoff = 32;
  int start = (int)(blockIdx.x % (unsigned)members);
  for (;;) {
    if (threadIdx.x < 32) {
      // warp 0 scans 32 members at a time (from this block's rotating start) for open
      // operations with items left; the candidate lanes then try, lowest first, to take
      // one: a ticket from the operation's own item counter (atomicAdd; a ticket past
      // the operation's items is simply dropped, and the counter is never reused, so
      // there are no compare-and-swap retries under contention).  The scan reads the
      // counters with plain volatile loads (an acquire load per member would invalidate
      // the SM's L1); the item taken is ordered after the release that opened it by one
      // acquire fence.
      const int lane = threadIdx.x;
      // one read of the error word, the same for every lane (the loop below and its
      // warp-wide ballots and shuffles must be uniform)
      int go = __shfl_sync(0xffffffffu, lane == 0 && ld_volatile(&st->err) != 0u ? -1 : 0, 0);
      int jo = 0, lt = 0;
      for (int base = 0; base < members && go == 0; base += 32) {
        const int k = base + lane;
        int j = 0, nt = 0;
        bool cand = false;
        if (k < members) {
          const int m = (start + k) % members;
          const int d = *reinterpret_cast<const volatile int*>(done + m);
          if (d < mops[m]) {
            j = mop0[m] + d;
            nt = ops[j].ntiles;
            cand = *reinterpret_cast<const volatile int*>(taken + j) < nt;
          }
        }
        unsigned mask = __ballot_sync(0xffffffffu, cand);
        while (mask != 0u && go == 0) {
          const int src = __ffs(mask) - 1;
          int got = 0, glt = 0;
          if (lane == src) {
            const int t = atomicAdd(taken + j, 1);
            if (t < nt) {
              got = 1;
              glt = t;
            }
          }
          if (__shfl_sync(0xffffffffu, got, src)) {
            go = 1;
            jo = __shfl_sync(0xffffffffu, j, src);
            lt = __shfl_sync(0xffffffffu, glt, src);
          }
          mask &= mask - 1u;
        }
      }
      if (lane == 0) {
        start = (start + 1) % members;
        if (go == 0) {
          if (ld_volatile(&st->finished) >= (unsigned)active) {
            go = -1;  // every member's chain is complete
          } else {
            const unsigned long long now = global_ns();
            if (idle_since == 0) idle_since = now;
            if (now - idle_since > wait_ns) {
              atomicOr(&st->err, 1u);
              go = -1;
            } else {
              __nanosleep(backoff);
              backoff = backoff < 512 ? 2 * backoff : 512;
            }
          }
        } else if (go > 0) {
          fence_acquire();
          idle_since = 0;
          backoff = 32;
        }
        s_go = go;
        s_op = jo;
        s_lt = lt;
      }
      start = __shfl_sync(0xffffffffu, start, 0);
    }
    __syncthreads();
    const int go = s_go;
    if (go < 0) break;
    if (go == 0) {
      __syncthreads();  // thread 0 rewrites s_* only after every thread has read them
      continue;
    }
    const POp& op = ops[s_op];
    const CfW<float>& w = wts[op.member];
    const int b0 = s_lt * op.per_tile;
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
      if (c == op.ntiles) {
        if (op.seq + 1 == mops[op.member]) atomicAdd(&st->finished, 1u);
        st_release(done + op.member, op.seq + 1);
      }
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

cudaError_t launch_persist(const POp* ops, const int* mop0, const int* mops, int members,
                           int active, const void* wts, PState* st, int* done, int* taken,
                           int* count, unsigned long long wait_ns, int grid, cudaStream_t s) {
  if (members < 1 || active < 1 || grid < 1) return cudaErrorInvalidValue;
  k_persist<<<grid, kPersistThreads, 0, s>>>(ops, mop0, mops, members, active,
                                             static_cast<const CfW<float>*>(wts), st, done,
                                             taken, count, wait_ns);
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

// Self-test of the bounded wait (no counterpart in the paper): a launch whose blocks
// are told to wait for a second hierarchy that has no work, so nothing ever opens;
// with a 100 ms limit the blocks give up, set the error word and the launch ends.
extern "C" mg_status mg_selftest_persist_wait(void) {
  using namespace mgk;
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };  // every region 256-aligned
  const size_t off_w = up(2 * sizeof(POp));
  const size_t off_z = up(off_w + persist_weight_bytes());
  const size_t off_s = up(off_z + 1024 * sizeof(float));
  const size_t off_d = up(off_s + sizeof(PState));  // done[2], taken[2 ops], count[2 ops]
  const size_t off_c = up(off_d + 6 * sizeof(int));  // mop0[2], mops[2]
  const size_t bytes = off_c + 4 * sizeof(int);
  char* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) return MG_ENOMEM;
  POp ops[2];
  std::memset(ops, 0, sizeof(ops));
  for (int q = 0; q < 2; ++q) {
    ops[q].kind = P_ZERO;
    ops[q].order = 2;
    ops[q].member = 0;
    ops[q].seq = q;
    ops[q].nblk = 1;
    ops[q].per_tile = 1;
    ops[q].ntiles = 1;
    ops[q].tile0 = q;
    ops[q].out0 = reinterpret_cast<float*>(d + off_z);
    ops[q].n = 1024;
  }
  // member 0 owns both operations; the launch is told that 2 members are active, so
  // after member 0's chain the blocks find nothing open and wait for a member that
  // never finishes: the wait must give up
  const int chain[4] = {0, 2, 2, 0};  // mop0[0..1], mops[0..1]
  std::vector<unsigned char> w(persist_weight_bytes(), 0);
  PState* st = reinterpret_cast<PState*>(d + off_s);
  int* done = reinterpret_cast<int*>(d + off_d);
  int* taken = done + 2;
  int* count = done + 4;
  const int* mop0 = reinterpret_cast<const int*>(d + off_c);
  cudaStream_t s = nullptr;
  mg_status r = MG_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMemcpyAsync(d, ops, sizeof(ops), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d + off_w, w.data(), w.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(d + off_s, 0, off_c - off_s, s) != cudaSuccess ||
      cudaMemcpyAsync(d + off_c, chain, sizeof(chain), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      launch_persist(reinterpret_cast<const POp*>(d), mop0, mop0 + 2, 2, 2, d + off_w, st, done,
                     taken, count, 100000000ull, 2, s) != cudaSuccess ||
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
