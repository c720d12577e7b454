// Hybrid Poisson solver correction (Hahn & Abel 2011, Sec. 3.5.2).
//
// The finite-difference solution loses small-scale power on the finest level; the
// paper replaces the finest level's own contribution by the exact k-space one:
// with f the level's source (zero outside the level, on a grid zero-padded to
// twice its size), the displacement correction is the difference between the
// exact gradient of the inverse Laplacian and the order-n finite-difference one,
//   d psi_j(k) = i [k_j / k^2 + g_j(k) / Lt(k)] f(k)
// for psi = -G phi, forward transform sum_x f(x) e^{-ik.x}, Lt = -sum_a lam_n(k_a h)
// / h^2 the Table 1 Laplacian symbol and i g_j = i g_n(k_j h) / h the Table 1
// gradient symbol (lam_2 = 2(1 - cos t), g_2 = sin t, and so on), 0 at k = 0 and,
// as the multiplier is odd in k_j, on the Nyquist plane of axis j.
// A single periodic level is corrected periodically, without padding.
//
// Steps: copy f into the (padded) real grid, cuFFT D2Z once; per component j a
// kernel forms the multiplied half spectrum (with the 1/N of the inverse), cuFFT
// Z2D, and a kernel adds the level's part of the result to psi_j.
#include <cufft.h>

#include "mg_internal.h"

namespace mgk {

namespace {

__device__ __forceinline__ void symbols(int order, double t, double& lam, double& g) {
  double s1, c1;
  sincos(t, &s1, &c1);
  if (order == 2) {
    lam = 2.0 * (1.0 - c1);
    g = s1;
    return;
  }
  double s2, c2;
  sincos(2.0 * t, &s2, &c2);
  if (order == 4) {
    lam = (c2 - 16.0 * c1 + 15.0) / 6.0;
    g = (8.0 * s1 - s2) / 6.0;
    return;
  }
  double s3, c3;
  sincos(3.0 * t, &s3, &c3);
  lam = (-2.0 * c3 + 27.0 * c2 - 270.0 * c1 + 245.0) / 90.0;
  g = (45.0 * s1 - 9.0 * s2 + s3) / 30.0;
}

// R (N0 x N1 x N2 dense) := f on [0, n) of every axis, 0 elsewhere.
__global__ void __launch_bounds__(256)
    k_pad(const double* __restrict__ f, int n0, int n1, int n2, double* __restrict__ R, int N0,
          int N1, int N2) {
  const long long total = (long long)N0 * N1 * N2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % N2);
    const long long r = e / N2;
    const int j = (int)(r % N1);
    const int i = (int)(r / N1);
    R[e] = (i < n0 && j < n1 && k < n2) ? __ldg(f + ((long long)i * n1 + j) * n2 + k) : 0.0;
  }
}

// W = i [k_j / k^2 + g_j / Lt] F / N over the half spectrum of the N grid.
__global__ void __launch_bounds__(256)
    k_hybrid_multiply(const cufftDoubleComplex* __restrict__ F, cufftDoubleComplex* __restrict__ W,
                      int N0, int N1, int N2, double h, int order, int comp) {
  const int N2h = N2 / 2 + 1;
  const long long total = (long long)N0 * N1 * N2h;
  const double pi2 = 2.0 * 3.14159265358979323846;
  const double inv_n = 1.0 / ((double)N0 * N1 * N2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e % N2h);
    const long long r = e / N2h;
    const int j = (int)(r % N1);
    const int i = (int)(r / N1);
    const int idx[3] = {i <= N0 / 2 ? i : i - N0, j <= N1 / 2 ? j : j - N1, m};
    const int NN[3] = {N0, N1, N2};
    double k[3], lam_sum = 0.0, ksq = 0.0, gc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double t = pi2 * (double)idx[a] / NN[a];  // k_a h
      k[a] = t / h;
      ksq += k[a] * k[a];
      double lam, g;
      symbols(order, t, lam, g);
      lam_sum += lam;
      if (a == comp) gc = g / h;
    }
    // the multiplier is odd in k_comp: 0 on the self-conjugate Nyquist plane of that
    // axis (even N), so the product stays Hermitian and its inverse real
    double c = 0.0;
    const bool nyq = (NN[comp] % 2 == 0) && idx[comp] == NN[comp] / 2;
    if (e != 0 && !nyq) {
      const double Lt = -lam_sum / (h * h);
      c = (k[comp] / ksq + gc / Lt) * inv_n;
    }
    const cufftDoubleComplex v = F[e];
    W[e] = make_cuDoubleComplex(-v.y * c, v.x * c);  // i c v
  }
}

// psi[x] += R[x] for x in the level's [0, n) block of the N grid.
__global__ void __launch_bounds__(256)
    k_crop_add(const double* __restrict__ R, int N1, int N2, double* __restrict__ psi, int n0,
               int n1, int n2) {
  const long long total = (long long)n0 * n1 * n2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % n2);
    const long long r = e / n2;
    const int j = (int)(r % n1);
    const int i = (int)(r / n1);
    psi[e] += __ldg(R + ((long long)i * N1 + j) * N2 + k);
  }
}

unsigned blocks_cap(long long work) {
  const long long b = (work + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

struct HybridFFT {
  int n[3] = {0, 0, 0}, N[3] = {0, 0, 0};
  double h = 0.0;
  int order = 2;
  double* R = nullptr;
  cufftDoubleComplex* F = nullptr;
  cufftDoubleComplex* W = nullptr;
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
};

size_t hybrid_bytes(int n0, int n1, int n2, bool pad) {
  const long long f = pad ? 2 : 1;
  const long long N0 = f * n0, N1 = f * n1, N2 = f * n2;
  const long long real = N0 * N1 * N2 * 8;
  const long long spec = N0 * N1 * (N2 / 2 + 1) * 16;
  // real grid, two half spectra, and about one half spectrum of cuFFT work area
  return (size_t)(real + 3 * spec);
}

void hybrid_destroy(HybridFFT* hy) {
  if (!hy) return;
  if (hy->have_fwd) cufftDestroy(hy->fwd);
  if (hy->have_inv) cufftDestroy(hy->inv);
  cudaFree(hy->R);
  cudaFree(hy->F);
  cudaFree(hy->W);
  delete hy;
}

cudaError_t hybrid_create(HybridFFT** out, int n0, int n1, int n2, double h, int order,
                          bool pad) {
  *out = nullptr;
  HybridFFT* hy = new HybridFFT();
  const int f = pad ? 2 : 1;
  hy->n[0] = n0;
  hy->n[1] = n1;
  hy->n[2] = n2;
  hy->N[0] = f * n0;
  hy->N[1] = f * n1;
  hy->N[2] = f * n2;
  hy->h = h;
  hy->order = order;
  const size_t real = (size_t)hy->N[0] * hy->N[1] * hy->N[2];
  const size_t spec = (size_t)hy->N[0] * hy->N[1] * (hy->N[2] / 2 + 1);
  cudaError_t e = cudaMalloc(&hy->R, real * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&hy->F, spec * sizeof(cufftDoubleComplex));
  if (e == cudaSuccess) e = cudaMalloc(&hy->W, spec * sizeof(cufftDoubleComplex));
  if (e == cudaSuccess) {
    if (cufftPlan3d(&hy->fwd, hy->N[0], hy->N[1], hy->N[2], CUFFT_D2Z) != CUFFT_SUCCESS) {
      e = cudaErrorMemoryAllocation;
    } else {
      hy->have_fwd = true;
      if (cufftPlan3d(&hy->inv, hy->N[0], hy->N[1], hy->N[2], CUFFT_Z2D) != CUFFT_SUCCESS)
        e = cudaErrorMemoryAllocation;
      else
        hy->have_inv = true;
    }
  }
  if (e != cudaSuccess) {
    hybrid_destroy(hy);
    return e;
  }
  *out = hy;
  return cudaSuccess;
}

cudaError_t hybrid_apply(HybridFFT* hy, const double* f, double* const psi[3], cudaStream_t s) {
  if (cufftSetStream(hy->fwd, s) != CUFFT_SUCCESS || cufftSetStream(hy->inv, s) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  const long long real = (long long)hy->N[0] * hy->N[1] * hy->N[2];
  const long long spec = (long long)hy->N[0] * hy->N[1] * (hy->N[2] / 2 + 1);
  const long long cells = (long long)hy->n[0] * hy->n[1] * hy->n[2];
  k_pad<<<blocks_cap(real), 256, 0, s>>>(f, hy->n[0], hy->n[1], hy->n[2], hy->R, hy->N[0],
                                         hy->N[1], hy->N[2]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (cufftExecD2Z(hy->fwd, hy->R, hy->F) != CUFFT_SUCCESS) return cudaErrorUnknown;
  for (int c = 0; c < 3; ++c) {
    k_hybrid_multiply<<<blocks_cap(spec), 256, 0, s>>>(hy->F, hy->W, hy->N[0], hy->N[1], hy->N[2],
                                                       hy->h, hy->order, c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (cufftExecZ2D(hy->inv, hy->W, hy->R) != CUFFT_SUCCESS) return cudaErrorUnknown;
    k_crop_add<<<blocks_cap(cells), 256, 0, s>>>(hy->R, hy->N[1], hy->N[2], psi[c], hy->n[0],
                                                 hy->n[1], hy->n[2]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace mgk
