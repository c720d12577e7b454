// Ghost zones (Hahn & Abel 2011, Sec. 3.2 periodic boundaries; Sec. 3.3
// coarse-fine boundaries).
//
// Coarse-fine faces of a nest, in three kernels:
//  * k_cf_tangential (once per parent state): for each face, each of the n/2
//    parent layers outside it and each fine tangential position, the degree-n
//    tensor Lagrange interpolant of the parent values parallel to the face
//    ("intermediate values"); and the part of the parent face flux (Table 2,
//    order n-1) that reads uncovered parent cells.
//  * k_cf_flux (before every half-sweep / residual): per parent face element,
//    the ghosts of its 4 fine columns from a degree-n polynomial normal to the
//    face through the n/2 intermediate values and n/2+1 fine interior values;
//    the parent flux with covered parent cells taken as the mean of their
//    current 8 children (two-way interface); the mean of the 4 fine fluxes;
//    and the difference added uniformly to the ghosts of each column so that
//    the fine fluxes average to the parent flux.
//  * k_cf_edges (before the 2LPT source only): edge and corner ghosts, which
//    only mixed derivatives read, by tensor degree-n interpolation of parent
//    values.
#include "mg_internal.h"
#include "mg_stencil.cuh"
#include "mg_vbody.cuh"

namespace mgk {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_ghost_periodic(Grid G, T* __restrict__ u) {
  ghost_periodic_body<T>(G, u, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <int ORDER, typename T>
__global__ void __launch_bounds__(128)
    k_cf_tangential(Grid F, Grid P, const T* __restrict__ pu, Int3 off, FaceSet fs, CfW<T> w,
                    T invH, T* __restrict__ inter, T* __restrict__ fc_unc) {
  cf_tangential_body<ORDER, T, Ldg>(F, P, pu, off, fs, w, invH, inter, fc_unc,
                                    blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <int ORDER, typename T>
__global__ void __launch_bounds__(128)
    k_cf_flux(Grid F, T* __restrict__ u, FaceSet fs, CfW<T> w, const T* __restrict__ inter,
              const T* __restrict__ fc_unc, T fc_scale, T a0, T a1, T b0, T b1, int flux_fix) {
  cf_flux_body<ORDER, T>(F, u, fs, w, inter, fc_unc, fc_scale, a0, a1, b0, b1, flux_fix,
                         blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <int ORDER, typename T>
__global__ void __launch_bounds__(128)
    k_cf_edges(Grid F, T* __restrict__ u, Grid P, const T* __restrict__ pu, Int3 off,
               CfWeights w) {
  constexpr int half = ORDER / 2;
  const int g = F.g;
  const int X = F.n0 + 2 * g, Y = F.n1 + 2 * g, Z = F.n2 + 2 * g;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)X * Y * Z) return;
  const int k = (int)(t % Z) - g;
  const int j = (int)((t / Z) % Y) - g;
  const int i = (int)(t / ((long long)Z * Y)) - g;
  const int out = (i < 0 || i >= F.n0) + (j < 0 || j >= F.n1) + (k < 0 || k >= F.n2);
  if (out < 2) return;
  const int pi = off.x + (i >> 1), pj = off.y + (j >> 1), pk = off.z + (k >> 1);
  const double* wi = w.tang[i & 1];
  const double* wj = w.tang[j & 1];
  const double* wk = w.tang[k & 1];
  T acc = T(0);
  for (int a = 0; a <= ORDER; ++a) {
    T pa = T(0);
    for (int bq = 0; bq <= ORDER; ++bq) {
      T row = T(0);
      for (int cq = 0; cq <= ORDER; ++cq)
        row = fma(T(wk[cq]), __ldg(pu + gidx(P, pi + a - half, pj + bq - half, pk + cq - half)), row);
      pa = fma(T(wj[bq]), row, pa);
    }
    acc = fma(T(wi[a]), pa, acc);
  }
  u[gidx(F, i, j, k)] = acc;
}

}  // namespace

template <typename T>
cudaError_t launch_ghost_periodic(const Grid& G, T* u, cudaStream_t s) {
  const long long g = G.g;
  const long long X = G.n0 + 2 * g, Y = G.n1 + 2 * g;
  const long long total = X * Y * 2 * g + X * 2 * g * G.n2 + 2 * g * (long long)G.n1 * G.n2;
  const int block = 256;
  k_ghost_periodic<T><<<(unsigned)((total + block - 1) / block), block, 0, s>>>(G, u);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cf_tangential(int order, const Grid& F, const Grid& P, const T* pu, Int3 off,
                                 const FaceSet& fs, const CfWeights& w, double invH, T* inter,
                                 T* fc_unc, cudaStream_t s) {
  const int block = 128;
  const unsigned grid = (unsigned)(((order / 2) * fs.ebase[6] + block - 1) / block);
  const CfW<T> wt = cf_weights_as<T>(w);
  switch (order) {
    case 2: k_cf_tangential<2, T><<<grid, block, 0, s>>>(F, P, pu, off, fs, wt, T(invH), inter, fc_unc); break;
    case 4: k_cf_tangential<4, T><<<grid, block, 0, s>>>(F, P, pu, off, fs, wt, T(invH), inter, fc_unc); break;
    case 6: k_cf_tangential<6, T><<<grid, block, 0, s>>>(F, P, pu, off, fs, wt, T(invH), inter, fc_unc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cf_flux(int order, const Grid& F, T* u, const FaceSet& fs, const CfWeights& w,
                           const T* inter, const T* fc_unc, double h, double invh, double invH,
                           int flux_fix, cudaStream_t s) {
  const int block = 128;
  const unsigned grid = (unsigned)((4 * fs.ebase[6] + block - 1) / block);
  const T fc_scale = T(0.125 * invH);
  const T a0 = T(h / w.ghost_coef[0]), a1 = T(h / w.ghost_coef[1]);
  const T b0 = T(0.25 * invh * h / w.ghost_coef[0]), b1 = T(0.25 * invh * h / w.ghost_coef[1]);
  const CfW<T> wt = cf_weights_as<T>(w);
  switch (order) {
    case 2: k_cf_flux<2, T><<<grid, block, 0, s>>>(F, u, fs, wt, inter, fc_unc, fc_scale, a0, a1, b0, b1, flux_fix); break;
    case 4: k_cf_flux<4, T><<<grid, block, 0, s>>>(F, u, fs, wt, inter, fc_unc, fc_scale, a0, a1, b0, b1, flux_fix); break;
    case 6: k_cf_flux<6, T><<<grid, block, 0, s>>>(F, u, fs, wt, inter, fc_unc, fc_scale, a0, a1, b0, b1, flux_fix); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cf_edges(int order, const Grid& F, T* u, const Grid& P, const T* pu, Int3 off,
                            const CfWeights& w, cudaStream_t s) {
  const long long total = (long long)(F.n0 + 2 * F.g) * (F.n1 + 2 * F.g) * (F.n2 + 2 * F.g);
  const int block = 128;
  const unsigned grid = (unsigned)((total + block - 1) / block);
  switch (order) {
    case 2: k_cf_edges<2, T><<<grid, block, 0, s>>>(F, u, P, pu, off, w); break;
    case 4: k_cf_edges<4, T><<<grid, block, 0, s>>>(F, u, P, pu, off, w); break;
    case 6: k_cf_edges<6, T><<<grid, block, 0, s>>>(F, u, P, pu, off, w); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#define MGK_GHOST_INSTANTIATE(T)                                                              \
  template cudaError_t launch_ghost_periodic<T>(const Grid&, T*, cudaStream_t);               \
  template cudaError_t launch_cf_tangential<T>(int, const Grid&, const Grid&, const T*, Int3, \
                                               const FaceSet&, const CfWeights&, double, T*,  \
                                               T*, cudaStream_t);                             \
  template cudaError_t launch_cf_flux<T>(int, const Grid&, T*, const FaceSet&,                \
                                         const CfWeights&, const T*, const T*, double,        \
                                         double, double, int, cudaStream_t);                  \
  template cudaError_t launch_cf_edges<T>(int, const Grid&, T*, const Grid&, const T*, Int3,  \
                                          const CfWeights&, cudaStream_t);

MGK_GHOST_INSTANTIATE(double)
MGK_GHOST_INSTANTIATE(float)

}  // namespace mgk
