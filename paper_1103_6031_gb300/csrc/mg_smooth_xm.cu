// Colour half-sweep of the smoother for float32 levels, with shared-memory plane tiles
// and an x-march (Hahn & Abel 2011, Sec. 3.2 smoothing step; the same update as
// k_smooth_half, bit-identical).
//
// A block of 32 x 8 threads owns 64 z-cells x 8 y-rows and marches through kXT planes
// along x.  Per plane, the block stages the plane's tile with its y and z halos
// (8 + 2 H rows x 72 elements, one float4 per thread) in shared memory (two buffers,
// one barrier per plane), so each update reads its y and z neighbours from shared
// memory instead of issuing a global load per neighbour; each thread keeps its own
// z-pair of planes i - H .. i + H in registers, so its x neighbours cost one float2
// load per plane.  The arithmetic and its order are those of k_smooth_half, and the
// output is the same: every interior cell of uout written (colour c updated, the other
// colour copied), ghost images on periodic levels.
//
// Used where the tiles fit without ragged edges: n0 a multiple of kXT, n1 of 8, n2 of
// 64, and the row layout of make_grid (interior at element 4 of a row, so the tile's
// first element, k = kt - 4, is 16-byte aligned).
#include "mg_internal.h"
#include "mg_stencil.cuh"

namespace mgk {

namespace {

constexpr int kXZ = 64;          // z-cells per tile (32 threads x 2)
constexpr int kXY = 8;           // y-rows per tile (one warp each)
constexpr int kXT = 4;           // planes per block
constexpr int kXW = kXZ + 8;     // staged elements per row: 4 on each side

// At least 4 blocks per SM (64 registers; 78 without the cap, 3 blocks per SM).
template <int ORDER>
__global__ void __launch_bounds__(32 * kXY, 4)
    k_smooth_half_xm(Grid G, const float* __restrict__ uin, float* __restrict__ uout,
                     const float* __restrict__ f, float a_f, int colour, int periodic) {
  constexpr int H = ORDER / 2;
  constexpr int R = kXY + 2 * H;     // staged rows
  constexpr int V4 = R * kXW / 4;    // float4 per staged tile
  __shared__ __align__(16) float tile[2][R * kXW];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int kt = blockIdx.x * kXZ, jt = blockIdx.y * kXY, i0 = blockIdx.z * kXT;
  const int k0 = kt + 2 * tx, j = jt + ty;
  const long long sy = G.Zp, sx = (long long)G.Y * G.Zp;
  // element of (plane i, row jt - H, z kt - 4): the tile's first element
  const long long tbase = gidx(G, 0, jt - H, kt - 4);
  const long long own = gidx(G, 0, j, k0);  // + i * sx: this thread's z-pair in plane i
  // x-queue: q[d] = this thread's pair in plane i - H + d
  float2 q[2 * H + 1];
#pragma unroll
  for (int d = 0; d < 2 * H; ++d)
    q[d] = *reinterpret_cast<const float2*>(uin + own + (long long)(i0 - H + d) * sx);
  const int cpos = (ty + H) * kXW + 4 + 2 * tx;  // this thread's pair in a staged tile
#pragma unroll
  for (int s = 0; s < kXT; ++s) {
    const int i = i0 + s;
    float* T = tile[s & 1];
    // stage plane i's tile: rows jt - H .. jt + kXY - 1 + H, z kt - 4 .. kt + 67
    for (int v = tid; v < V4; v += 32 * kXY) {
      const int r = v / (kXW / 4), c = v % (kXW / 4);
      *reinterpret_cast<float4*>(T + r * kXW + 4 * c) =
          *reinterpret_cast<const float4*>(uin + tbase + (long long)i * sx + r * sy + 4 * c);
    }
    q[2 * H] = *reinterpret_cast<const float2*>(uin + own + (long long)(i + H) * sx);
    __syncthreads();
    const int upd = (((i + j + k0) & 1) == colour) ? 0 : 1;
    const float* C = T + cpos + upd;  // the updated cell in the tile
    auto comp = [&](const float2& p) { return upd ? p.y : p.x; };
    // neighbour sums in k_smooth_half's order: (z) + (y) + (x)
    float s1 = (C[-1] + C[1]) + (C[-kXW] + C[kXW]) + (comp(q[H - 1]) + comp(q[H + 1]));
    float s2 = 0.f, s3 = 0.f;
    if (ORDER >= 4)
      s2 = (C[-2] + C[2]) + (C[-2 * kXW] + C[2 * kXW]) + (comp(q[H - 2]) + comp(q[H + 2]));
    if (ORDER >= 6)
      s3 = (C[-3] + C[3]) + (C[-3 * kXW] + C[3 * kXW]) + (comp(q[H - 3]) + comp(q[H + 3]));
    constexpr double wc = 3.0 * Lap<ORDER>::w0;
    const long long p0 = own + (long long)i * sx;
    float v = a_f * __ldg(f + p0 + upd);
    v = fmaf(float(-Lap<ORDER>::w1 / wc), s1, v);
    if (ORDER >= 4) v = fmaf(float(-Lap<ORDER>::w2 / wc), s2, v);
    if (ORDER >= 6) v = fmaf(float(-Lap<ORDER>::w3 / wc), s3, v);
    float2 out = q[H];
    if (upd) out.y = v;
    else out.x = v;
    *reinterpret_cast<float2*>(uout + p0) = out;
    if (periodic) write_pair_images<float>(G, uout, i, j, k0, out.x, out.y);
#pragma unroll
    for (int d = 0; d < 2 * H; ++d) q[d] = q[d + 1];
  }
}

}  // namespace

bool smooth_xm_usable(const Grid& G) {
  return G.za == 4 && G.n0 % kXT == 0 && G.n1 % kXY == 0 && G.n2 % kXZ == 0;
}

cudaError_t launch_smooth_half_xm(int order, const Grid& G, const float* uin, float* uout,
                                  const float* f, double a_f, int colour, int periodic,
                                  cudaStream_t s) {
  if (!smooth_xm_usable(G)) return cudaErrorInvalidValue;
  dim3 block(32, kXY, 1);
  dim3 grid(G.n2 / kXZ, G.n1 / kXY, G.n0 / kXT);
  switch (order) {
    case 2: k_smooth_half_xm<2><<<grid, block, 0, s>>>(G, uin, uout, f, float(a_f), colour, periodic); break;
    case 4: k_smooth_half_xm<4><<<grid, block, 0, s>>>(G, uin, uout, f, float(a_f), colour, periodic); break;
    case 6: k_smooth_half_xm<6><<<grid, block, 0, s>>>(G, uin, uout, f, float(a_f), colour, periodic); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mgk
