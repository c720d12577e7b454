// Colour half-sweep of the smoother through TMA-staged plane tiles (Hahn & Abel
// 2011, Sec. 3.2 smoothing step; the same update as k_smooth_half).
//
// A block owns a tile of 64 z-cells x 8 y-rows and marches along x over a chunk
// of 8 planes (fully unrolled: slots, phases and queue positions are static).  One elected thread streams the planes of u (with their y and z
// halos of width order/2) into a ring of shared-memory slots with
// cp.async.bulk.tensor, several planes ahead of the computation; every slot has
// an mbarrier that completes when its bytes have landed.  Each thread keeps the
// 2*order/2+1 values of its own z-pair along x in registers (a sliding queue),
// so the x neighbours cost nothing, and reads its y and z neighbours from the
// centre plane's slot.  The planes of f that the block updates (interior rows
// only) travel in the same slots, under the same mbarrier, so no global load
// is left on the critical path; the result pair is stored coalesced.
//
// The arithmetic, its order and the output (colour c updated, the other colour
// copied, ghost images on periodic levels) are those of k_smooth_half, so the two
// kernels give bit-identical results.
//
// Every wait on an mbarrier is bounded (kWaitNs of global time); a block whose
// wait ran out sets *err, stops, drains its copies in flight (again bounded) and
// returns, so a lost copy surfaces as an error status instead of a hang.  Blocks
// that are still waiting give up as soon as *err is set (and later launches on the
// same flag fail fast), so the whole launch ends within about one wait limit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mg_internal.h"
#include "mg_stencil.cuh"

namespace mgk {

namespace {

constexpr int kTZ = 64;       // cells along z per tile: 32 lanes x 2
constexpr int kTY = 8;        // rows along y per tile: one warp each
constexpr int kBZ = kTZ + 8;  // staged elements per row: 4 halo elements on each side
constexpr int kSlots = 8;     // plane tiles per block (in flight + in use)
constexpr int kLX = 8;        // planes updated per block (the march is fully unrolled)
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

template <typename T, int H>
struct Tile {
  static constexpr int BY = kTY + 2 * H;                  // staged rows of u
  static constexpr int elems = kBZ * BY;                  // elements per u box
  static constexpr int bytes = elems * (int)sizeof(T);    // bytes per u box
  static constexpr int f_off = (bytes + 127) / 128 * 128 / (int)sizeof(T);  // f box in a slot
  static constexpr int f_bytes = kTZ * kTY * (int)sizeof(T);  // bytes per f box
  static constexpr int stride_bytes = f_off * (int)sizeof(T) + f_bytes;
  static constexpr int stride = stride_bytes / (int)sizeof(T);
  static constexpr int smem = kSlots * stride_bytes;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void proxy_async_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// true once the phase with this parity has completed; false after kWaitNs, or as
// soon as *stop is non-zero (another block of the launch gave up already, so a lost
// copy surfaces after about one wait limit rather than one per block wave); stop may
// be null (the drain of a failing block waits for its own copies regardless)
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          const unsigned* stop) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitNs) return false;
    if (stop && *reinterpret_cast<const volatile unsigned*>(stop) != 0u) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_plane(void* dst, const CUtensorMap* tm, int cz, int cy,
                                               int cx, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(cz), "r"(cy), "r"(cx),
      "r"(smem_addr(bar))
      : "memory");
}

template <int ORDER, typename T>
__global__ void __launch_bounds__(32 * kTY)
    k_smooth_half_tma(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tf,
                      Grid G, T* __restrict__ uout, T a_f, int colour, int periodic,
                      unsigned* __restrict__ err, unsigned extra_tx) {
  constexpr int H = ORDER / 2;
  constexpr int NT = kLX + 2 * H;  // planes staged by a block with a full chunk
  static_assert(kSlots >= 2 * H + 1 && kSlots <= NT, "slot ring too small or too large");
  typedef Tile<T, H> TL;
  typedef typename Vec2<T>::type V2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tiles = reinterpret_cast<T*>(smem_raw);
  __shared__ __align__(8) unsigned long long bar[kSlots];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int kt = blockIdx.x * kTZ;
  const int jt = blockIdx.y * kTY;
  const int i0 = blockIdx.z * kLX;
  const int nu = min(kLX, G.n0 - i0);  // planes i0 .. i0+nu-1 are updated
  const int nt = nu + 2 * H;           // staged planes: t = 0 .. nt-1 is plane i0 - H + t
  const int k = kt + 2 * tx;           // first cell of this thread's z-pair
  const int j = jt + ty;
  const bool active = j < G.n1 && k < G.n2;
  const bool pair = k + 1 < G.n2;
  const bool issuer = tx == 0 && ty == 0;
  // u box origin: element za + kt - 4 of the row (a multiple of 4 elements, so the
  // first copied byte is 16-byte aligned), row jt - H; f box: element za + kt, row jt
  const int cz = kt + G.za - 4;
  const int cy = jt + G.g - H;
  const int cx = i0 - H + G.g;  // plane coordinate of t = 0
  // periodic levels: only cells within g of a face have ghost images
  const bool yz_face = k < G.g || k + 1 >= G.n2 - G.g || j < G.g || j >= G.n1 - G.g;

  if (issuer) {
#pragma unroll
    for (int s = 0; s < kSlots; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncthreads();

  int next = 0;  // issuer: staged planes t < next have been issued
  // plane t of u (with halos) into slot t % kSlots, and of f when the block updates it
  auto issue = [&](int t) {
    next = t + 1;
    T* dst = tiles + (t % kSlots) * TL::stride;
    unsigned long long* b = &bar[t % kSlots];
    const bool fpl = t >= H && t < H + nu;
    // extra_tx (0 except in the wait-limit self-test) keeps plane 0's phase open
    mbar_expect_tx(b, (unsigned)(TL::bytes + (fpl ? TL::f_bytes : 0)) + (t == 0 ? extra_tx : 0u));
    tma_load_plane(dst, &tin, cz, cy, cx + t, b);
    if (fpl) tma_load_plane(dst + TL::f_off, &tf, kt + G.za, jt + G.g, cx + t, b);
  };
  if (issuer) {
    proxy_async_fence();
#pragma unroll
    for (int t = 0; t < kSlots; ++t)
      if (t < nt) issue(t);
  }

  // this thread's pair within a slot: row ty + H, element 4 + 2 tx; its f: row ty
  const int own = (ty + H) * kBZ + 4 + 2 * tx;
  const int fown = TL::f_off + ty * kTZ + 2 * tx;
  int waited = 0;  // staged planes t < waited have been waited for
  bool bad = false;
  V2 q[NT];  // q[t]: this thread's pair in staged plane t
#pragma unroll
  for (int t = 0; t < 2 * H; ++t) {
    bad |= !mbar_wait(&bar[t % kSlots], (t / kSlots) & 1, err);
    q[t] = *reinterpret_cast<const V2*>(tiles + (t % kSlots) * TL::stride + own);
  }
  waited = 2 * H;
  // planes t < H only fed the queue: their slots take the next planes
  if (__syncthreads_or(bad)) goto fail;
  if (issuer) {
    proxy_async_fence();
#pragma unroll
    for (int t = kSlots; t < kSlots + H; ++t)
      if (t < nt) issue(t);
  }

  {
    const long long sx = (long long)G.Y * G.Zp;
    T* orow = uout + gidx(G, i0, j, k);
    const int base = ((i0 + j) ^ colour) & 1;  // updated cell of the pair in plane i0
#pragma unroll
    for (int s = 0; s < kLX; ++s) {
      if (s < nu) {
        const int tq = s + 2 * H;  // plane entering the queue
        bad |= !mbar_wait(&bar[tq % kSlots], (tq / kSlots) & 1, err);
        q[tq] = *reinterpret_cast<const V2*>(tiles + (tq % kSlots) * TL::stride + own);
        waited = tq + 1;
        if (active) {
          const int tc = s + H;  // centre plane i = i0 + s
          const T* C = tiles + (tc % kSlots) * TL::stride + own;
          const int upd = base ^ (s & 1);
          const V2 c = q[tc];
          // z neighbours of the updated cell: pairs at -2 and +2 and one more value
          const V2 zl = *reinterpret_cast<const V2*>(C - 2);
          const V2 zr = *reinterpret_cast<const V2*>(C + 2);
          const T zm1 = upd ? c.x : zl.y;
          const T zp1 = upd ? zr.x : c.y;
          const T zm2 = upd ? zl.y : zl.x;
          const T zp2 = upd ? zr.y : zr.x;
          T zm3 = T(0), zp3 = T(0);
          if constexpr (ORDER >= 6) {
            const T far = C[upd ? 4 : -3];
            zm3 = upd ? zl.x : far;
            zp3 = upd ? far : zr.y;
          }
          const T* Cu = C + upd;
          auto comp = [&](const V2& v) { return upd ? v.y : v.x; };  // the updated cell's value
          T s1 = (zm1 + zp1) + (Cu[-kBZ] + Cu[kBZ]) + (comp(q[tc - 1]) + comp(q[tc + 1]));
          T s2 = T(0), s3 = T(0);
          if constexpr (ORDER >= 4)
            s2 = (zm2 + zp2) + (Cu[-2 * kBZ] + Cu[2 * kBZ]) + (comp(q[tc - 2]) + comp(q[tc + 2]));
          if constexpr (ORDER >= 6)
            s3 = (zm3 + zp3) + (Cu[-3 * kBZ] + Cu[3 * kBZ]) + (comp(q[tc - 3]) + comp(q[tc + 3]));
          constexpr double wc = 3.0 * Lap<ORDER>::w0;
          T v = a_f * tiles[(tc % kSlots) * TL::stride + fown + upd];
          v = fma(T(-Lap<ORDER>::w1 / wc), s1, v);
          if constexpr (ORDER >= 4) v = fma(T(-Lap<ORDER>::w2 / wc), s2, v);
          if constexpr (ORDER >= 6) v = fma(T(-Lap<ORDER>::w3 / wc), s3, v);
          T* o = orow + s * sx;
          const int i = i0 + s;
          const bool img = periodic && (yz_face || i < G.g || i >= G.n0 - G.g);
          if (pair) {
            V2 out = c;
            if (upd) out.y = v; else out.x = v;
            *reinterpret_cast<V2*>(o) = out;
            if (img) write_pair_images<T>(G, uout, i, j, k, out.x, out.y);
          } else {
            // lone last cell of an odd row: updated only when it has the colour
            const T ov = upd ? c.x : v;
            *o = ov;
            if (img) write_images<T>(G, uout, i, j, k, ov);
          }
        }
        // every thread is done with the centre plane's slot: it takes plane
        // s + H + kSlots
        if (__syncthreads_or(bad)) goto fail;
        const int tn = s + H + kSlots;
        if (issuer && tn < nt) {
          proxy_async_fence();
          issue(tn);
        }
      }
    }
  }
  return;

fail:
  // drain the copies this block issued and has not waited for, then report
  if (issuer) {
    for (int t = waited; t < next; ++t) mbar_wait(&bar[t % kSlots], (t / kSlots) & 1, nullptr);
    atomicOr(err, 1u);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <int ORDER, typename T>
cudaError_t launch_order(const Grid& G, const CUtensorMap* tin, const CUtensorMap* tf, T* uout,
                         T a_f, int colour, int periodic, unsigned* err, unsigned extra_tx,
                         cudaStream_t s) {
  typedef Tile<T, ORDER / 2> TL;
  dim3 block(32, kTY, 1);
  dim3 grid((G.n2 + kTZ - 1) / kTZ, (G.n1 + kTY - 1) / kTY, (G.n0 + kLX - 1) / kLX);
  k_smooth_half_tma<ORDER, T><<<grid, block, TL::smem, s>>>(*tin, *tf, G, uout, a_f, colour,
                                                            periodic, err, extra_tx);
  return cudaGetLastError();
}

template <int ORDER, typename T>
cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(k_smooth_half_tma<ORDER, T>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, Tile<T, ORDER / 2>::smem);
}

}  // namespace

bool smooth_tma_usable(const Grid& G) { return G.za == 4 && encode_fn() != nullptr; }

cudaError_t prepare_smooth_tma() {
  cudaError_t e = cudaSuccess;
  cudaError_t r;
  if ((r = set_smem_attr<2, float>()) != cudaSuccess) e = r;
  if ((r = set_smem_attr<4, float>()) != cudaSuccess) e = r;
  if ((r = set_smem_attr<6, float>()) != cudaSuccess) e = r;
  if ((r = set_smem_attr<2, double>()) != cudaSuccess) e = r;
  if ((r = set_smem_attr<4, double>()) != cudaSuccess) e = r;
  if ((r = set_smem_attr<6, double>()) != cudaSuccess) e = r;
  return e;
}

cudaError_t make_plane_tmap(const Grid& G, const void* base, int elem_bytes, int order,
                            bool halo, CUtensorMap* tm) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc || (elem_bytes != 4 && elem_bytes != 8) || (reinterpret_cast<size_t>(base) & 15))
    return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {(cuuint64_t)G.Zp, (cuuint64_t)G.Y, (cuuint64_t)G.X};
  const cuuint64_t strides[2] = {(cuuint64_t)G.Zp * elem_bytes,
                                 (cuuint64_t)G.Zp * G.Y * elem_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)(halo ? kBZ : kTZ),
                             (cuuint32_t)(halo ? kTY + order : kTY), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r =
      enc(tm, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
          3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_smooth_half_tma(int order, const Grid& G, const CUtensorMap* tin,
                                   const CUtensorMap* tf, T* uout, double a_f, int colour,
                                   int periodic, unsigned* err, cudaStream_t s,
                                   unsigned extra_tx) {
  if (G.za != 4) return cudaErrorInvalidValue;
  switch (order) {
    case 2: return launch_order<2, T>(G, tin, tf, uout, T(a_f), colour, periodic, err, extra_tx, s);
    case 4: return launch_order<4, T>(G, tin, tf, uout, T(a_f), colour, periodic, err, extra_tx, s);
    case 6: return launch_order<6, T>(G, tin, tf, uout, T(a_f), colour, periodic, err, extra_tx, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_smooth_half_tma<float>(int, const Grid&, const CUtensorMap*,
                                                   const CUtensorMap*, float*, double, int, int,
                                                   unsigned*, cudaStream_t, unsigned);
template cudaError_t launch_smooth_half_tma<double>(int, const Grid&, const CUtensorMap*,
                                                    const CUtensorMap*, double*, double, int, int,
                                                    unsigned*, cudaStream_t, unsigned);

}  // namespace mgk
