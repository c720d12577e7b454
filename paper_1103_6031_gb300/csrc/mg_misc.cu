// Coarsest-level solve, convergence norms, composite mean, packing between the
// caller's dense arrays and the padded level layout, the 2LPT source and the
// displacement gradient (Hahn & Abel 2011, Sec. 3.1, 3.2).
#include "mg_internal.h"
#include "mg_stencil.cuh"
#include "mg_vbody.cuh"

namespace mgk {

namespace {

// Table 1 gradient: antisymmetric weights on offsets +1, +2, +3 (units 1/h).
template <int ORDER>
struct Grad;
template <>
struct Grad<2> {
  static constexpr double g1 = 0.5, g2 = 0.0, g3 = 0.0;
};
template <>
struct Grad<4> {
  static constexpr double g1 = 8.0 / 12.0, g2 = -1.0 / 12.0, g3 = 0.0;
};
template <>
struct Grad<6> {
  static constexpr double g1 = 45.0 / 60.0, g2 = -9.0 / 60.0, g3 = 1.0 / 60.0;
};

template <int ORDER>
__device__ __forceinline__ double grad_w(int s) {  // weight at offset s in [-3, 3]
  const int a = s < 0 ? -s : s;
  const double v = a == 1 ? Grad<ORDER>::g1 : (a == 2 ? Grad<ORDER>::g2 : (a == 3 ? Grad<ORDER>::g3 : 0.0));
  return s < 0 ? -v : v;
}

template <int ORDER>
__device__ __forceinline__ double lap_w(int s) {
  const int a = s < 0 ? -s : s;
  return a == 0 ? Lap<ORDER>::w0 : (a == 1 ? Lap<ORDER>::w1 : (a == 2 ? Lap<ORDER>::w2 : Lap<ORDER>::w3));
}

// Periodic pseudo-inverse of L on the coarsest level as a circular convolution:
// u(x) = sum_y K(x - y) f(y), K precomputed on the host from the DFT symbol.
// One block per output cell; the block's threads split the sum over y.  The
// result is also written to the cell's periodic ghost images.
constexpr int kCoarseBlock = kCoarseThreads;

template <typename T>
__global__ void __launch_bounds__(kCoarseBlock)
    k_coarsest(Grid G, const T* __restrict__ f, T* __restrict__ u,
               const double* __restrict__ kern) {
  coarsest_body<T, Ldg>(G, f, u, kern, (int)blockIdx.x, (int)threadIdx.x);
}

template <int BLOCK>
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[BLOCK], sb[BLOCK];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
#pragma unroll
  for (int w = BLOCK / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  a = sa[0];
  b = sb[0];
}

constexpr int kRedBlock = 256;

// One block per (x plane, 8 y rows); 32 lanes stride along z.  Block b writes
// its partial sums to slot b, so the reduction order is fixed.
// With r32 != nullptr the float64 residual of every uncovered interior cell is also
// stored, rounded to float32, as the source of the correction equation (mixed
// precision); covered cells are skipped for both.
template <int ORDER>
__global__ void __launch_bounds__(kRedBlock)
    k_norm_partial(Grid G, const double* __restrict__ u, const double* __restrict__ f,
                   double invh2, double vol, Int3 clo, Int3 chi, double* __restrict__ partial,
                   float* __restrict__ r32) {
  const long long sy = G.Zp, sx = (long long)G.Y * G.Zp;
  const int i = blockIdx.y;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  double rr = 0.0, ff = 0.0;
  if (j < G.n1) {
    const bool row_cov = i >= clo.x && i < chi.x && j >= clo.y && j < chi.y;
    const long long row = gidx(G, i, j, 0);
    for (int k = lane; k < G.n2; k += 32) {
      // covered cells: no norm term, and no correction source either (the FAS
      // restriction overwrites a covered parent cell's source before the parent uses it)
      const bool cov = row_cov && k >= clo.z && k < chi.z;
      if (cov) continue;
      const long long p = row + k;
      const double fv = __ldg(f + p);
      const double r = u ? fma(-invh2, lap_h2<ORDER, double>(u, p, sy, sx), fv) : fv;
      if (r32) r32[p] = (float)r;
      rr = fma(r, r, rr);
      ff = fma(fv, fv, ff);
    }
  }
  block_sum2<kRedBlock>(rr, ff);
  if (threadIdx.x == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    partial[2 * b] = rr * vol;
    partial[2 * b + 1] = ff * vol;
  }
}

__global__ void __launch_bounds__(kRedBlock)
    k_sum_partial(Grid G, const double* __restrict__ f, double vol, Int3 clo, Int3 chi,
                  double* __restrict__ partial) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  double s = 0.0, unused = 0.0;
  if (j < G.n1) {
    const bool row_cov = i >= clo.x && i < chi.x && j >= clo.y && j < chi.y;
    const long long row = gidx(G, i, j, 0);
    for (int k = lane; k < G.n2; k += 32) {
      if (row_cov && k >= clo.z && k < chi.z) continue;
      s += __ldg(f + row + k);
    }
  }
  block_sum2<kRedBlock>(s, unused);
  if (threadIdx.x == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    partial[2 * b] = s * vol;
    partial[2 * b + 1] = 0.0;
  }
}

// Sums `count` consecutive (a, b) pairs in a fixed order into out[0], out[1].
__global__ void __launch_bounds__(kRedBlock)
    k_reduce_partials(const double* __restrict__ partial, int count, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < count; t += kRedBlock) {
    a += partial[2 * t];
    b += partial[2 * t + 1];
  }
  block_sum2<kRedBlock>(a, b);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// Block 0: exactly k_reduce_partials over all `count` pairs into out[0], out[1].
// Block 1 + l: the pairs of leaf level l alone, [R.off[l], R.off[l] + R.cnt[l]), into
// out_levels[2 l], out_levels[2 l + 1] (the per-level residual and source sums).
__global__ void __launch_bounds__(kRedBlock)
    k_reduce_levels(const double* __restrict__ partial, int count, LevelRanges R,
                    double* __restrict__ out, double* __restrict__ out_levels) {
  int lo = 0, hi = count;
  if (blockIdx.x > 0) {
    lo = R.off[blockIdx.x - 1];
    hi = lo + R.cnt[blockIdx.x - 1];
  }
  double a = 0.0, b = 0.0;
  for (int t = lo + threadIdx.x; t < hi; t += kRedBlock) {
    a += partial[2 * t];
    b += partial[2 * t + 1];
  }
  block_sum2<kRedBlock>(a, b);
  if (threadIdx.x == 0) {
    double* o = blockIdx.x == 0 ? out : out_levels + 2 * (blockIdx.x - 1);
    o[0] = a;
    o[1] = b;
  }
}

__global__ void __launch_bounds__(256)
    k_pack(Grid G, const double* __restrict__ src, double* __restrict__ dst, double shift) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= n) return;
  const int k = (int)(t % G.n2), j = (int)((t / G.n2) % G.n1), i = (int)(t / ((long long)G.n2 * G.n1));
  dst[gidx(G, i, j, k)] = __ldg(src + t) - shift;
}

__global__ void __launch_bounds__(256)
    k_unpack(Grid G, const double* __restrict__ src, double* __restrict__ dst, double add) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= n) return;
  const int k = (int)(t % G.n2), j = (int)((t / G.n2) % G.n1), i = (int)(t / ((long long)G.n2 * G.n1));
  dst[t] = __ldg(src + gidx(G, i, j, k)) + add;
}

// f -= mean, f2 = f on the interior; mean = *mean_num * inv_volume (device-side).
__global__ void __launch_bounds__(256)
    k_shift_copy(Grid G, double* __restrict__ f, double* __restrict__ f2,
                 const double* __restrict__ mean_num, double inv_volume) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= n) return;
  const int k = (int)(t % G.n2), j = (int)((t / G.n2) % G.n1), i = (int)(t / ((long long)G.n2 * G.n1));
  const long long p = gidx(G, i, j, k);
  const double v = f[p] - mean_num[0] * inv_volume;
  f[p] = v;
  if (f2) f2[p] = v;
}

// u += e on the interior (float64 += float32 correction); periodic levels also
// update their ghost images.  One thread per cell of a (32 x 4)-cell tile row.
__global__ void __launch_bounds__(128)
    k_add_correction(Grid G, double* __restrict__ u, const float* __restrict__ e, int periodic) {
  const int k = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 4 + threadIdx.y;
  const int i = blockIdx.z;
  if (k >= G.n2 || j >= G.n1) return;
  const long long p = gidx(G, i, j, k);
  const double v = u[p] + (double)__ldg(e + p);
  u[p] = v;
  if (periodic) write_images<double>(G, u, i, j, k, v);
}

// p -= sum[0] * scale over n elements (sum read on the device).
__global__ void __launch_bounds__(256)
    k_sub_mean(double* __restrict__ p, long long n, const double* __restrict__ sum, double scale) {
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t < n) p[t] -= sum[0] * scale;
}

__global__ void __launch_bounds__(256) k_fill(double* __restrict__ p, long long n, double v) {
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t < n) p[t] = v;
}

// First derivatives D_b = G_b phi (Table 1 gradient, times h) for the 2LPT
// source, on every cell whose b coordinate is interior and whose other two
// coordinates lie anywhere in the ghost-padded box (the mixed derivatives read
// D_b up to g cells outside the interior along the other axes).  One thread per
// (padded x, padded y) row position, looping over padded z.
template <int ORDER>
__global__ void __launch_bounds__(128)
    k_first_derivs(Grid G, const double* __restrict__ phi, double* __restrict__ dx,
                   double* __restrict__ dy, double* __restrict__ dz) {
  constexpr int half = ORDER / 2;
  const int g = G.g;
  const int k = (int)(blockIdx.x * 32 + threadIdx.x) - g;
  const int j = (int)(blockIdx.y * 4 + threadIdx.y) - g;
  const int i = (int)blockIdx.z - g;
  if (k >= G.n2 + g || j >= G.n1 + g) return;
  const long long p = gidx(G, i, j, k);
  const long long st[3] = {(long long)G.Y * G.Zp, (long long)G.Zp, 1};
  const int crd[3] = {i, j, k};
  const int n[3] = {G.n0, G.n1, G.n2};
  double* out[3] = {dx, dy, dz};
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (crd[b] < 0 || crd[b] >= n[b]) continue;
    double acc = 0.0;
#pragma unroll
    for (int s = 1; s <= half; ++s)
      acc = fma(grad_w<ORDER>(s), __ldg(phi + p + s * st[b]) - __ldg(phi + p - s * st[b]), acc);
    out[b][p] = acc;
  }
}

// Finite-difference Hessian at element p: d[a] = phi_aa, the 1D second difference
// along a; m = (phi_xy, phi_xz, phi_yz), phi_ab = G_a (G_b phi) from the stored
// first derivatives.
template <int ORDER>
__device__ __forceinline__ void fd_hessian(const Grid& G, const double* __restrict__ phi,
                                           const double* __restrict__ dy,
                                           const double* __restrict__ dz, double invh2,
                                           long long p, double (&d)[3], double (&m)[3]) {
  constexpr int half = ORDER / 2;
  const long long st[3] = {(long long)G.Y * G.Zp, (long long)G.Zp, 1};
  const double c = __ldg(phi + p);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double acc = Lap<ORDER>::w0 * c;
#pragma unroll
    for (int s = 1; s <= half; ++s)
      acc = fma(lap_w<ORDER>(s), __ldg(phi + p + s * st[a]) + __ldg(phi + p - s * st[a]), acc);
    d[a] = acc * invh2;
  }
  // phi_xy = G_x D_y, phi_xz = G_x D_z, phi_yz = G_y D_z
  const double* src[3] = {dy, dz, dz};
  const int ax[3] = {0, 0, 1};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double acc = 0.0;
#pragma unroll
    for (int s = 1; s <= half; ++s)
      acc = fma(grad_w<ORDER>(s), __ldg(src[q] + p + s * st[ax[q]]) - __ldg(src[q] + p - s * st[ax[q]]),
                acc);
    m[q] = acc * invh2;
  }
}

// tau = sum_{i<j} (phi_ii phi_jj - phi_ij^2) (Sec. 3.1.2).
template <int ORDER>
__global__ void __launch_bounds__(128)
    k_lpt2_source(Grid G, const double* __restrict__ phi, const double* __restrict__ dx,
                  const double* __restrict__ dy, const double* __restrict__ dz, double invh2,
                  double* __restrict__ tau) {
  const int k = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 4 + threadIdx.y;
  const int i = blockIdx.z;
  if (k >= G.n2 || j >= G.n1) return;
  const long long p = gidx(G, i, j, k);
  double d[3], m[3];
  fd_hessian<ORDER>(G, phi, dy, dz, invh2, p, d, m);
  tau[p] = fma(d[0], d[1] + d[2], d[1] * d[2]) - fma(m[0], m[0], fma(m[1], m[1], m[2] * m[2]));
}

// Local Lagrangian density (Sec. 5.3): with H the Hessian of the combined
// potential Phi (L = -grad Phi), rho / rho_bar = 1 / det[I - H]; writes
// 1/det - 1 (the renormalisation and the +1 follow on the host side).
// det[I - H] = a b c - a m_yz^2 - b m_xz^2 - c m_xy^2 - 2 m_xy m_xz m_yz with
// a, b, c = 1 - phi_xx, 1 - phi_yy, 1 - phi_zz.
template <int ORDER>
__global__ void __launch_bounds__(128)
    k_lla(Grid G, const double* __restrict__ phi, const double* __restrict__ dy,
          const double* __restrict__ dz, double invh2, double* __restrict__ out) {
  const int k = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 4 + threadIdx.y;
  const int i = blockIdx.z;
  if (k >= G.n2 || j >= G.n1) return;
  const long long p = gidx(G, i, j, k);
  double d[3], m[3];
  fd_hessian<ORDER>(G, phi, dy, dz, invh2, p, d, m);
  const double a = 1.0 - d[0], b = 1.0 - d[1], c = 1.0 - d[2];
  const double det = a * b * c - a * m[2] * m[2] - b * m[1] * m[1] - c * m[0] * m[0] -
                     2.0 * m[0] * m[1] * m[2];
  out[p] = 1.0 / det - 1.0;
}

// out[t] = a1 x1[t] + a2 x2[t] (x2 may be NULL) over n dense elements.
__global__ void __launch_bounds__(256)
    k_axpby(long long n, double a1, const double* __restrict__ x1, double a2,
            const double* __restrict__ x2, double* __restrict__ out) {
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= n) return;
  out[t] = x2 ? fma(a2, __ldg(x2 + t), a1 * __ldg(x1 + t)) : a1 * __ldg(x1 + t);
}

template <int ORDER>
__global__ void __launch_bounds__(128)
    k_gradient(Grid G, const double* __restrict__ phi, double invh, double* __restrict__ dx,
               double* __restrict__ dy, double* __restrict__ dz) {
  constexpr int half = ORDER / 2;
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const long long t = blockIdx.x * 128LL + threadIdx.x;
  if (t >= n) return;
  const int k = (int)(t % G.n2), j = (int)((t / G.n2) % G.n1), i = (int)(t / ((long long)G.n2 * G.n1));
  const long long p = gidx(G, i, j, k);
  const long long st[3] = {(long long)G.Y * G.Zp, (long long)G.Zp, 1};
  double out[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double acc = 0.0;
#pragma unroll
    for (int s = 1; s <= half; ++s)
      acc = fma(grad_w<ORDER>(s), __ldg(phi + p + s * st[a]) - __ldg(phi + p - s * st[a]), acc);
    out[a] = -acc * invh;
  }
  dx[t] = out[0];
  dy[t] = out[1];
  dz[t] = out[2];
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

int norm_blocks(const Grid& G) { return ((G.n1 + 7) / 8) * G.n0; }

cudaError_t launch_coarsest(const Grid& G, const double* f, double* u, const double* kern,
                            cudaStream_t s) {
  const int n = G.n0 * G.n1 * G.n2;
  k_coarsest<double><<<n, kCoarseBlock, 0, s>>>(G, f, u, kern);
  return cudaGetLastError();
}

cudaError_t launch_coarsest(const Grid& G, const float* f, float* u, const double* kern,
                            cudaStream_t s) {
  const int n = G.n0 * G.n1 * G.n2;
  k_coarsest<float><<<n, kCoarseBlock, 0, s>>>(G, f, u, kern);
  return cudaGetLastError();
}

cudaError_t launch_norm_partial(int order, const Grid& G, const double* u, const double* f,
                                double invh2, double vol, Int3 clo, Int3 chi, double* partial,
                                int blocks, float* r32, cudaStream_t s) {
  const dim3 grid((G.n1 + 7) / 8, G.n0);
  if ((int)(grid.x * grid.y) != blocks) return cudaErrorInvalidValue;
  switch (order) {
    case 2: k_norm_partial<2><<<grid, kRedBlock, 0, s>>>(G, u, f, invh2, vol, clo, chi, partial, r32); break;
    case 4: k_norm_partial<4><<<grid, kRedBlock, 0, s>>>(G, u, f, invh2, vol, clo, chi, partial, r32); break;
    case 6: k_norm_partial<6><<<grid, kRedBlock, 0, s>>>(G, u, f, invh2, vol, clo, chi, partial, r32); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sum_partial(const Grid& G, const double* f, double vol, Int3 clo, Int3 chi,
                               double* partial, int blocks, cudaStream_t s) {
  const dim3 grid((G.n1 + 7) / 8, G.n0);
  if ((int)(grid.x * grid.y) != blocks) return cudaErrorInvalidValue;
  k_sum_partial<<<grid, kRedBlock, 0, s>>>(G, f, vol, clo, chi, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partial, int count, int width, double* out,
                                   cudaStream_t s) {
  (void)width;
  k_reduce_partials<<<1, kRedBlock, 0, s>>>(partial, count, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_levels(const double* partial, int count, const LevelRanges& R,
                                 double* out, double* out_levels, cudaStream_t s) {
  if (R.n < 0 || R.n > MG_MAX_LEVELS) return cudaErrorInvalidValue;
  for (int l = 0; l < R.n; ++l)
    if (R.off[l] < 0 || R.cnt[l] < 0 || R.off[l] + R.cnt[l] > count) return cudaErrorInvalidValue;
  k_reduce_levels<<<1 + R.n, kRedBlock, 0, s>>>(partial, count, R, out, out_levels);
  return cudaGetLastError();
}

cudaError_t launch_pack(const Grid& G, const double* src, double* dst, double shift,
                        cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  k_pack<<<blocks_for(n, 256), 256, 0, s>>>(G, src, dst, shift);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const Grid& G, const double* src, double* dst, cudaStream_t s,
                          double add) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  k_unpack<<<blocks_for(n, 256), 256, 0, s>>>(G, src, dst, add);
  return cudaGetLastError();
}

cudaError_t launch_shift_copy(const Grid& G, double* f, double* f2, const double* mean_num,
                              double inv_volume, cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  k_shift_copy<<<blocks_for(n, 256), 256, 0, s>>>(G, f, f2, mean_num, inv_volume);
  return cudaGetLastError();
}

cudaError_t launch_add_correction(const Grid& G, double* u, const float* e, int periodic,
                                  cudaStream_t s) {
  dim3 block(32, 4, 1);
  dim3 grid((G.n2 + 31) / 32, (G.n1 + 3) / 4, G.n0);
  k_add_correction<<<grid, block, 0, s>>>(G, u, e, periodic);
  return cudaGetLastError();
}

cudaError_t launch_sub_mean(double* p, long long n, const double* sum, double scale,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_sub_mean<<<blocks_for(n, 256), 256, 0, s>>>(p, n, sum, scale);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill<<<blocks_for(n, 256), 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t launch_lpt2_source(int order, const Grid& G, const double* phi, double invh2,
                               double* tau, double* work, cudaStream_t s) {
  const long long e = grid_elems(G);
  double* dx = work;
  double* dy = work + e;
  double* dz = work + 2 * e;
  const dim3 block(32, 4, 1);
  const dim3 gpad((G.n2 + 2 * G.g + 31) / 32, (G.n1 + 2 * G.g + 3) / 4, G.n0 + 2 * G.g);
  const dim3 gin((G.n2 + 31) / 32, (G.n1 + 3) / 4, G.n0);
  switch (order) {
    case 2:
      k_first_derivs<2><<<gpad, block, 0, s>>>(G, phi, dx, dy, dz);
      k_lpt2_source<2><<<gin, block, 0, s>>>(G, phi, dx, dy, dz, invh2, tau);
      break;
    case 4:
      k_first_derivs<4><<<gpad, block, 0, s>>>(G, phi, dx, dy, dz);
      k_lpt2_source<4><<<gin, block, 0, s>>>(G, phi, dx, dy, dz, invh2, tau);
      break;
    case 6:
      k_first_derivs<6><<<gpad, block, 0, s>>>(G, phi, dx, dy, dz);
      k_lpt2_source<6><<<gin, block, 0, s>>>(G, phi, dx, dy, dz, invh2, tau);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_lla(int order, const Grid& G, const double* phi, double invh2, double* out,
                       double* work, cudaStream_t s) {
  const long long e = grid_elems(G);
  double* dx = work;
  double* dy = work + e;
  double* dz = work + 2 * e;
  const dim3 block(32, 4, 1);
  const dim3 gpad((G.n2 + 2 * G.g + 31) / 32, (G.n1 + 2 * G.g + 3) / 4, G.n0 + 2 * G.g);
  const dim3 gin((G.n2 + 31) / 32, (G.n1 + 3) / 4, G.n0);
  switch (order) {
    case 2:
      k_first_derivs<2><<<gpad, block, 0, s>>>(G, phi, dx, dy, dz);
      k_lla<2><<<gin, block, 0, s>>>(G, phi, dy, dz, invh2, out);
      break;
    case 4:
      k_first_derivs<4><<<gpad, block, 0, s>>>(G, phi, dx, dy, dz);
      k_lla<4><<<gin, block, 0, s>>>(G, phi, dy, dz, invh2, out);
      break;
    case 6:
      k_first_derivs<6><<<gpad, block, 0, s>>>(G, phi, dx, dy, dz);
      k_lla<6><<<gin, block, 0, s>>>(G, phi, dy, dz, invh2, out);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_axpby(long long n, double a1, const double* x1, double a2, const double* x2,
                         double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_axpby<<<blocks_for(n, 256), 256, 0, s>>>(n, a1, x1, a2, x2, out);
  return cudaGetLastError();
}

cudaError_t launch_gradient(int order, const Grid& G, const double* phi, double invh, double* dx,
                            double* dy, double* dz, cudaStream_t s) {
  const long long n = (long long)G.n0 * G.n1 * G.n2;
  const unsigned b = blocks_for(n, 128);
  switch (order) {
    case 2: k_gradient<2><<<b, 128, 0, s>>>(G, phi, invh, dx, dy, dz); break;
    case 4: k_gradient<4><<<b, 128, 0, s>>>(G, phi, invh, dx, dy, dz); break;
    case 6: k_gradient<6><<<b, 128, 0, s>>>(G, phi, invh, dx, dy, dz); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mgk
