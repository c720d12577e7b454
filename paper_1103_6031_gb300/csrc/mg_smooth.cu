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

template <typename T>
cudaError_t launch_smooth_half(int order, const Grid& G, const T* uin, T* uout, const T* f,
                               double a_f, int colour, int periodic, int rows, cudaStream_t s) {
  if (rows < 1 || rows > 8) return cudaErrorInvalidValue;
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
                                             int, int, int, cudaStream_t);                     \
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
