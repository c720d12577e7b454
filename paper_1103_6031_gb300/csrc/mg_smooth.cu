// Red-black Gauss-Seidel half-sweeps, residual + restriction, FAS source and
// prolongation-correction (Hahn & Abel 2011, Sec. 3.2 steps 2-9; Sec. 3.3).
//
// Smoother: one colour c = (i+j+k) mod 2 per launch.  Every cell of colour c
// takes the value that solves its own row of L u = f with all other values
// fixed at their pre-half-sweep values ("colour-Jacobi"; exact red-black GS for
// the 7-point stencil; for 13/19 points same-colour cells at distance 2 couple
// and this fixes their order).  The kernel reads buffer `uin` and writes every
// interior cell of `uout` (colour c updated, the other colour copied), so no
// thread ever reads a value another thread of the same launch writes.
#include "mg_internal.h"
#include "mg_stencil.cuh"
#include "mg_vbody.cuh"

namespace mgk {

namespace {

constexpr int kPairX = kVPairX;  // z-pairs per block row; blockDim.y = rows (1..8)
// At least 5 blocks of up to 256 threads per SM: caps the smoother at 48 registers
// (80 unbounded).  Measured on GB300 in CUDA graphs: float32 half-sweeps 15-20%
// faster at 128^3 (more warps in flight for the L1-bound loads), float64 unchanged
// (bound by the FP64 pipe).
#ifndef MG_SMOOTH_MIN_BLOCKS
#define MG_SMOOTH_MIN_BLOCKS 5
#endif

template <int ORDER, typename T>
__global__ void __launch_bounds__(kPairX * 8, MG_SMOOTH_MIN_BLOCKS)
    k_smooth_half(Grid G, const T* __restrict__ uin, T* __restrict__ uout,
                  const T* __restrict__ f, T a_f, int colour, int periodic) {
  smooth_half_body<ORDER, T, Ldg>(G, uin, uout, f, a_f, colour, periodic, (int)blockDim.y,
                                  Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                                      (int)threadIdx.x, (int)threadIdx.y});
}

// float32 rows whose length is a multiple of 4: one z-quad per thread (elements k0 ..
// k0 + 3, 16-byte aligned: the first interior element of a row sits at index 4 and the
// row pitch is a multiple of 8), updating the quad's two cells of colour c.  Every
// neighbour row along x and y is one 16-byte load serving both updates, and the z
// window k0 - 4 .. k0 + 7 three more; the two cells' sums and updates are those of
// smooth_half_body term by term, so the result is bit-identical to it.  The colour
// offset (0 or 1) is a run-time value shared by a row: it picks operands by select,
// never by a dynamic index into a register array.
__device__ __forceinline__ float4 ld4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

template <int ORDER>
__global__ void __launch_bounds__(256, 4)
    k_smooth_quad(Grid G, const float* __restrict__ uin, float* __restrict__ uout,
                  const float* __restrict__ f, float a_f, int colour, int periodic) {
  constexpr int R = ORDER / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = blockIdx.z;
  const int k0 = 4 * t;
  if (j >= G.n1 || k0 >= G.n2) return;
  const long long sy = G.Zp;
  const long long sx = (long long)G.Y * G.Zp;
  const long long p0 = gidx(G, i, j, k0);
  // the quad's cells of colour c are k0 + o and k0 + o + 2
  const bool o = ((i + j) & 1) != colour;
  const float4 c = ld4(uin + p0);
  float w[12];  // z window: elements k0 - 4 .. k0 + 7
  {
    const float4 a = ld4(uin + p0 - 4), b = ld4(uin + p0 + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = c.x; w[5] = c.y; w[6] = c.z; w[7] = c.w;
    w[8] = b.x; w[9] = b.y; w[10] = b.z; w[11] = b.w;
  }
  // x and y neighbours at distance d of the two updated cells: [cell][d - 1]
  float xm[2][R], xp[2][R], ym[2][R], yp[2][R];
#pragma unroll
  for (int d = 1; d <= R; ++d) {
    const float4 a = ld4(uin + p0 - d * sx), b = ld4(uin + p0 + d * sx);
    const float4 e = ld4(uin + p0 - d * sy), g = ld4(uin + p0 + d * sy);
    xm[0][d - 1] = o ? a.y : a.x; xm[1][d - 1] = o ? a.w : a.z;
    xp[0][d - 1] = o ? b.y : b.x; xp[1][d - 1] = o ? b.w : b.z;
    ym[0][d - 1] = o ? e.y : e.x; ym[1][d - 1] = o ? e.w : e.z;
    yp[0][d - 1] = o ? g.y : g.x; yp[1][d - 1] = o ? g.w : g.z;
  }
  const float4 fv = ld4(f + p0);
  const float fc[2] = {o ? fv.y : fv.x, o ? fv.w : fv.z};
  constexpr double wc = 3.0 * Lap<ORDER>::w0;
  float v[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    // z neighbour at offset q of cell k0 + 2h + o: window index 4 + 2h + o + q
#define MGK_ZN(q) (o ? w[5 + 2 * h + (q)] : w[4 + 2 * h + (q)])
    const float s1 = (MGK_ZN(-1) + MGK_ZN(1)) + (ym[h][0] + yp[h][0]) + (xm[h][0] + xp[h][0]);
    float r = a_f * fc[h];
    r = fmaf(float(-Lap<ORDER>::w1 / wc), s1, r);
    if constexpr (ORDER >= 4) {
      const float s2 = (MGK_ZN(-2) + MGK_ZN(2)) + (ym[h][1] + yp[h][1]) + (xm[h][1] + xp[h][1]);
      r = fmaf(float(-Lap<ORDER>::w2 / wc), s2, r);
    }
    if constexpr (ORDER >= 6) {
      const float s3 = (MGK_ZN(-3) + MGK_ZN(3)) + (ym[h][2] + yp[h][2]) + (xm[h][2] + xp[h][2]);
      r = fmaf(float(-Lap<ORDER>::w3 / wc), s3, r);
    }
#undef MGK_ZN
    v[h] = r;
  }
  float4 out = c;
  if (o) {
    out.y = v[0];
    out.w = v[1];
  } else {
    out.x = v[0];
    out.z = v[1];
  }
  *reinterpret_cast<float4*>(uout + p0) = out;
  if (periodic) {
    write_pair_images<float>(G, uout, i, j, k0, out.x, out.y);
    write_pair_images<float>(G, uout, i, j, k0 + 2, out.z, out.w);
  }
}

// One thread per covered parent cell: r = f - L u at its 8 children,
// parent u := mean(u), ubar := mean(u), parent f_fas := mean(r) (L ubar added later).
template <int ORDER, typename T>
__global__ void __launch_bounds__(128)
    k_residual_restrict(Grid F, const T* __restrict__ u, const T* __restrict__ f, T invh2, Grid P,
                        T* __restrict__ pu, T* __restrict__ pfas, T* __restrict__ ubar, Int3 off,
                        Int3 cn, int parent_periodic) {
  residual_restrict_body<ORDER, T, Ldg>(F, u, f, invh2, P, pu, pfas, ubar, off, cn,
                                        parent_periodic,
                                        Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                                            (int)threadIdx.x, (int)threadIdx.y});
}

// Covered parent cells: f_fas += L u (u = restricted fine solution there).
template <int ORDER, typename T>
__global__ void __launch_bounds__(128)
    k_fas_source(Grid P, const T* __restrict__ pu, T* __restrict__ pfas, T invH2, Int3 off,
                 Int3 cn) {
  fas_source_body<ORDER, T, Ldg>(P, pu, pfas, invH2, off, cn,
                                 Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                                     (int)threadIdx.x, (int)threadIdx.y});
}

// u += inject(parent u - ubar) on the fine interior; one thread per z-pair.
template <typename T>
__global__ void __launch_bounds__(128)
    k_prolong(Grid F, T* __restrict__ u, Grid P, const T* __restrict__ pu,
              const T* __restrict__ ubar, Int3 off, Int3 cn, int periodic) {
  prolong_body<T, Ldg>(F, u, P, pu, ubar, off, cn, periodic,
                       Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)threadIdx.x,
                           (int)threadIdx.y});
}

// parent u := mean of children (covered region), one thread per parent cell.
template <typename T>
__global__ void __launch_bounds__(128)
    k_restrict_u(Grid F, const T* __restrict__ u, Grid P, T* __restrict__ pu, Int3 off, Int3 cn) {
  const int kc = blockIdx.x * blockDim.x + threadIdx.x;
  const int jc = blockIdx.y * blockDim.y + threadIdx.y;
  const int ic = blockIdx.z;
  if (kc >= cn.z || jc >= cn.y) return;
  T s = T(0);
#pragma unroll
  for (int di = 0; di < 2; ++di)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
      typedef typename Vec2<T>::type V2;
      const V2 v = *reinterpret_cast<const V2*>(u + gidx(F, 2 * ic + di, 2 * jc + dj, 2 * kc));
      s += v.x + v.y;
    }
  pu[gidx(P, off.x + ic, off.y + jc, off.z + kc)] = s * T(0.125);
}

dim3 coarse_grid(Int3 cn, dim3 block) {
  return dim3((cn.z + block.x - 1) / block.x, (cn.y + block.y - 1) / block.y, cn.x);
}

}  // namespace

// The z-quad kernel: as many threads per block as the pair kernel's (32 x rows), the
// block's x extent the row's quads up to 32.
cudaError_t launch_smooth_quad(int order, const Grid& G, const float* uin, float* uout,
                               const float* f, double a_f, int colour, int periodic, int rows,
                               cudaStream_t s) {
  const int quads = G.n2 / 4;
  const int qx = quads < 32 ? quads : 32;
  int by = 32 * rows / qx;
  if (by > G.n1) by = G.n1;
  dim3 block(qx, by, 1);
  dim3 grid((quads + qx - 1) / qx, (G.n1 + by - 1) / by, G.n0);
  switch (order) {
    case 2: k_smooth_quad<2><<<grid, block, 0, s>>>(G, uin, uout, f, float(a_f), colour, periodic); break;
    case 4: k_smooth_quad<4><<<grid, block, 0, s>>>(G, uin, uout, f, float(a_f), colour, periodic); break;
    case 6: k_smooth_quad<6><<<grid, block, 0, s>>>(G, uin, uout, f, float(a_f), colour, periodic); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth_half(int order, const Grid& G, const T* uin, T* uout, const T* f,
                               double a_f, int colour, int periodic, int rows, bool quad,
                               cudaStream_t s) {
  if (rows < 1 || rows > 8) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (quad && G.n2 % 4 == 0 && G.n2 > 0 && G.n1 > 0)
      return launch_smooth_quad(order, G, uin, uout, f, a_f, colour, periodic, rows, s);
  }
  dim3 block(kPairX, rows, 1);
  const int pairs = (G.n2 + 1) / 2;
  dim3 grid((pairs + kPairX - 1) / kPairX, (G.n1 + rows - 1) / rows, G.n0);
  switch (order) {
    case 2: k_smooth_half<2, T><<<grid, block, 0, s>>>(G, uin, uout, f, T(a_f), colour, periodic); break;
    case 4: k_smooth_half<4, T><<<grid, block, 0, s>>>(G, uin, uout, f, T(a_f), colour, periodic); break;
    case 6: k_smooth_half<6, T><<<grid, block, 0, s>>>(G, uin, uout, f, T(a_f), colour, periodic); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_restrict(int order, const Grid& F, const T* u, const T* f,
                                     double invh2, const Grid& P, T* pu, T* pfas, T* ubar,
                                     Int3 off, Int3 cn, int parent_periodic, cudaStream_t s) {
  dim3 block(32, 4, 1);
  dim3 grid = coarse_grid(cn, block);
  switch (order) {
    case 2: k_residual_restrict<2, T><<<grid, block, 0, s>>>(F, u, f, T(invh2), P, pu, pfas, ubar, off, cn, parent_periodic); break;
    case 4: k_residual_restrict<4, T><<<grid, block, 0, s>>>(F, u, f, T(invh2), P, pu, pfas, ubar, off, cn, parent_periodic); break;
    case 6: k_residual_restrict<6, T><<<grid, block, 0, s>>>(F, u, f, T(invh2), P, pu, pfas, ubar, off, cn, parent_periodic); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fas_source(int order, const Grid& P, const T* pu, T* pfas, double invH2,
                              Int3 off, Int3 cn, cudaStream_t s) {
  dim3 block(32, 4, 1);
  dim3 grid = coarse_grid(cn, block);
  switch (order) {
    case 2: k_fas_source<2, T><<<grid, block, 0, s>>>(P, pu, pfas, T(invH2), off, cn); break;
    case 4: k_fas_source<4, T><<<grid, block, 0, s>>>(P, pu, pfas, T(invH2), off, cn); break;
    case 6: k_fas_source<6, T><<<grid, block, 0, s>>>(P, pu, pfas, T(invH2), off, cn); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(const Grid& F, T* u, const Grid& P, const T* pu, const T* ubar,
                           Int3 off, Int3 cn, int periodic, cudaStream_t s) {
  dim3 block(32, 4, 1);
  const int pairs = F.n2 / 2;
  dim3 grid((pairs + 31) / 32, (F.n1 + 3) / 4, F.n0);
  k_prolong<T><<<grid, block, 0, s>>>(F, u, P, pu, ubar, off, cn, periodic);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict_u(const Grid& F, const T* u, const Grid& P, T* pu, Int3 off, Int3 cn,
                              cudaStream_t s) {
  dim3 block(32, 4, 1);
  dim3 grid = coarse_grid(cn, block);
  k_restrict_u<T><<<grid, block, 0, s>>>(F, u, P, pu, off, cn);
  return cudaGetLastError();
}

#define MGK_INSTANTIATE(T)                                                                     \
  template cudaError_t launch_smooth_half<T>(int, const Grid&, const T*, T*, const T*, double, \
                                             int, int, int, bool, cudaStream_t);               \
  template cudaError_t launch_residual_restrict<T>(int, const Grid&, const T*, const T*,       \
                                                   double, const Grid&, T*, T*, T*, Int3,      \
                                                   Int3, int, cudaStream_t);                   \
  template cudaError_t launch_fas_source<T>(int, const Grid&, const T*, T*, double, Int3,      \
                                            Int3, cudaStream_t);                               \
  template cudaError_t launch_prolong<T>(const Grid&, T*, const Grid&, const T*, const T*,     \
                                         Int3, Int3, int, cudaStream_t);                       \
  template cudaError_t launch_restrict_u<T>(const Grid&, const T*, const Grid&, T*, Int3,      \
                                            Int3, cudaStream_t);

MGK_INSTANTIATE(double)
MGK_INSTANTIATE(float)

}  // namespace mgk
