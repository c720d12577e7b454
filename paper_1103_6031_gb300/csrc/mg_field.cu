// Density generator (Hahn & Abel 2011, Sec. 2.1): Gaussian white noise from a
// counter-based generator and its periodic convolution with a radial amplitude,
// delta = IFFT[A(|k|) FFT[noise]].
//
// Noise: Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011) written from its
// definition: counter (q mod 2^32, q div 2^32, 0, 0) for pair index q, key (seed
// mod 2^32, seed div 2^32); 10 rounds of two 32x32->64-bit products with the
// constants 0xD2511F53 and 0xCD9E8D57, the high halves mixed with the other two
// counter words and the key, the key bumped by 0x9E3779B9 and 0xBB67AE85 before
// every round but the first.  The four outputs give two uniforms in (0, 1) of 53
// bits each (27 + 26 bits plus half a unit in the last place) and two normal
// deviates by the Box-Muller transform: elements 2q and 2q + 1 of the noise.
//
// Field: cuFFT real-to-complex transform of the noise, a kernel that multiplies
// every mode by A(|k|) / N (linear interpolation of a table sampled at |k| = t dk,
// 0 beyond the table and at k = 0), and the complex-to-real inverse.
#include <cufft.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "mg.h"

namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t (&x)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * x[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * x[2];
    const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x[1] ^ k0;
    const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = (uint32_t)p1;
    x[2] = y2;
    x[3] = (uint32_t)p0;
  }
}

__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

// One Philox call per pair of elements; grid-stride over pairs.  stream is counter
// word 2 (0 for a single field, the level of a nest in the multi-scale field).
__global__ void __launch_bounds__(256)
    k_white_noise(unsigned long long seed, unsigned stream, long long n, double* __restrict__ out) {
  const long long pairs = (n + 1) / 2;
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < pairs;
       q += (long long)gridDim.x * blockDim.x) {
    uint32_t x[4] = {(uint32_t)((unsigned long long)q & 0xFFFFFFFFull),
                     (uint32_t)((unsigned long long)q >> 32), stream, 0u};
    philox4x32_10(x, k0, k1);
    const double u1 = uniform53(x[0], x[1]);
    const double u2 = uniform53(x[2], x[3]);
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    const long long i = 2 * q;
    if (i + 1 < n) {
      *reinterpret_cast<double2*>(out + i) = make_double2(r * c, r * s);
    } else {
      out[i] = r * c;
    }
  }
}

// F[i][j][m] *= A(|k|) * scale, m < n2/2 + 1 (half spectrum along z).
__global__ void __launch_bounds__(256)
    k_apply_amplitude(cufftDoubleComplex* __restrict__ F, int n0, int n1, int n2, double h,
                      const double* __restrict__ amp, int nt, double dk, double scale) {
  const int n2h = n2 / 2 + 1;
  const long long total = (long long)n0 * n1 * n2h;
  const double tp = 2.0 * 3.14159265358979323846 / h;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e % n2h);
    const long long r = e / n2h;
    const int j = (int)(r % n1);
    const int i = (int)(r / n1);
    const double fi = (double)(i <= n0 / 2 ? i : i - n0) / n0;
    const double fj = (double)(j <= n1 / 2 ? j : j - n1) / n1;
    const double fm = (double)m / n2;
    const double kmag = tp * sqrt(fi * fi + fj * fj + fm * fm);
    const double t = kmag / dk;
    double a = 0.0;
    if (t <= (double)(nt - 1)) {
      int it = (int)t;
      if (it > nt - 2) it = nt - 2;
      a = amp[it] + (t - it) * (amp[it + 1] - amp[it]);
    }
    if (e == 0) a = 0.0;
    a *= scale;
    F[e].x *= a;
    F[e].y *= a;
  }
}

int grid_for(long long work) {
  long long b = (work + 255) / 256;
  const long long cap = 152 * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ---- multi-scale field on a nested hierarchy (Sec. 2.3) ------------------------

#define GRID_STRIDE(e, total)                                                  \
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (total); \
       e += (long long)gridDim.x * blockDim.x)

// Hoffman-Ribak (Sec. 2.3.1): the mean of the 8 children of every parent cell of the
// nest region becomes parent / sqrt(8).  One thread per parent cell.
__global__ void __launch_bounds__(256)
    k_hoffman_ribak(double* __restrict__ own, int n0, int n1, int n2,
                    const double* __restrict__ parent, int P1, int P2, int o0, int o1, int o2) {
  const int c0n = n0 / 2, c1n = n1 / 2, c2n = n2 / 2;
  GRID_STRIDE(e, (long long)c0n * c1n * c2n) {
    const int c2 = (int)(e % c2n);
    const long long r = e / c2n;
    const int c1 = (int)(r % c1n);
    const int c0 = (int)(r / c1n);
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          sum += own[((long long)(2 * c0 + a) * n1 + 2 * c1 + b) * n2 + 2 * c2 + c];
    const double target =
        parent[((long long)(o0 + c0) * P1 + o1 + c1) * P2 + o2 + c2] / sqrt(8.0);
    const double shift = target - sum * 0.125;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          own[((long long)(2 * c0 + a) * n1 + 2 * c1 + b) * n2 + 2 * c2 + c] += shift;
  }
}

// R (N grid) := src on [0, n), with the box [lo, hi) of src zeroed, 0 elsewhere.
__global__ void __launch_bounds__(256)
    k_mask_pad(const double* __restrict__ src, int n0, int n1, int n2, double* __restrict__ R,
               int N0, int N1, int N2, int l0, int l1, int l2, int h0, int h1, int h2) {
  GRID_STRIDE(e, (long long)N0 * N1 * N2) {
    const int k = (int)(e % N2);
    const long long r = e / N2;
    const int j = (int)(r % N1);
    const int i = (int)(r / N1);
    double v = 0.0;
    if (i < n0 && j < n1 && k < n2 &&
        !(i >= l0 && i < h0 && j >= l1 && j < h1 && k >= l2 && k < h2))
      v = src[((long long)i * n1 + j) * n2 + k];
    R[e] = v;
  }
}

// dst (n grid) := R[0:n) (+ add, when add is not NULL).
__global__ void __launch_bounds__(256)
    k_crop(const double* __restrict__ R, int N1, int N2, double* __restrict__ dst, int n0, int n1,
           int n2, const double* __restrict__ add) {
  GRID_STRIDE(e, (long long)n0 * n1 * n2) {
    const int k = (int)(e % n2);
    const long long r = e / n2;
    const int j = (int)(r % n1);
    const int i = (int)(r / n1);
    const double v = R[((long long)i * N1 + j) * N2 + k];
    dst[e] = add ? v + add[e] : v;
  }
}

// Conservative tricubic interpolation of a parent-level field onto the nest (Sec.
// 2.3.3-2.3.4): each fine value is the tensor cubic Lagrange interpolation through the
// 4 nearest parent cells along every axis (nodes -1, 0, 1, 2 from the first node; the
// fine centre at t = 3/4 for an even index, 1/4 for an odd one); the 8 children of
// a parent cell are then shifted by a common amount so they average to the parent
// value.  One thread per parent cell of the nest region.
__global__ void __launch_bounds__(128)
    k_tricubic(const double* __restrict__ parent, int P1, int P2, int o0, int o1, int o2,
               double* __restrict__ fine, int n0, int n1, int n2) {
  // Lagrange weights at t = 3/4 (even fine index) and t = 1/4 (odd), nodes -1..2
  double wt[2][4];
#pragma unroll
  for (int par = 0; par < 2; ++par) {
    const double t = par ? 0.25 : 0.75;
    wt[par][0] = -t * (t - 1.0) * (t - 2.0) / 6.0;
    wt[par][1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
    wt[par][2] = -(t + 1.0) * t * (t - 2.0) / 2.0;
    wt[par][3] = (t + 1.0) * t * (t - 1.0) / 6.0;
  }
  const int c0n = n0 / 2, c1n = n1 / 2, c2n = n2 / 2;
  GRID_STRIDE(e, (long long)c0n * c1n * c2n) {
    const int c2 = (int)(e % c2n);
    const long long r = e / c2n;
    const int c1 = (int)(r % c1n);
    const int c0 = (int)(r / c1n);
    double val[8];
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          // first node: parent index - 2 for an even child, - 1 for an odd one
          const int f0 = o0 + c0 - 2 + a, f1 = o1 + c1 - 2 + b, f2 = o2 + c2 - 2 + c;
          double acc0 = 0.0;
          for (int s0 = 0; s0 < 4; ++s0) {
            double acc1 = 0.0;
            for (int s1 = 0; s1 < 4; ++s1) {
              const double* row = parent + ((long long)(f0 + s0) * P1 + f1 + s1) * P2 + f2;
              double acc2 = 0.0;
#pragma unroll
              for (int s2 = 0; s2 < 4; ++s2) acc2 = fma(wt[c][s2], row[s2], acc2);
              acc1 = fma(wt[b][s1], acc2, acc1);
            }
            acc0 = fma(wt[a][s0], acc1, acc0);
          }
          val[(a * 2 + b) * 2 + c] = acc0;
          sum += acc0;
        }
    const double shift =
        parent[((long long)(o0 + c0) * P1 + o1 + c1) * P2 + o2 + c2] - sum * 0.125;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          fine[((long long)(2 * c0 + a) * n1 + 2 * c1 + b) * n2 + 2 * c2 + c] =
              val[(a * 2 + b) * 2 + c] + shift;
  }
}

// parent[o + c] := mean of its 8 children in fine (covered cells).
__global__ void __launch_bounds__(256)
    k_children_mean_into(const double* __restrict__ fine, int n0, int n1, int n2,
                         double* __restrict__ parent, int P1, int P2, int o0, int o1, int o2) {
  const int c0n = n0 / 2, c1n = n1 / 2, c2n = n2 / 2;
  GRID_STRIDE(e, (long long)c0n * c1n * c2n) {
    const int c2 = (int)(e % c2n);
    const long long r = e / c2n;
    const int c1 = (int)(r % c1n);
    const int c0 = (int)(r / c1n);
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          sum += fine[((long long)(2 * c0 + a) * n1 + 2 * c1 + b) * n2 + 2 * c2 + c];
    parent[((long long)(o0 + c0) * P1 + o1 + c1) * P2 + o2 + c2] = sum * 0.125;
  }
}

// One periodic convolution of R (N grid) in place: D2Z, A(|k|) * scale, Z2D.
mg_status convolve_grid(const int N[3], double h, const double* amp, int nt, double dk,
                        double* R, cufftDoubleComplex* F, cudaStream_t s) {
  cufftHandle fwd, inv;
  if (cufftPlan3d(&fwd, N[0], N[1], N[2], CUFFT_D2Z) != CUFFT_SUCCESS) return MG_ECUDA;
  if (cufftPlan3d(&inv, N[0], N[1], N[2], CUFFT_Z2D) != CUFFT_SUCCESS) {
    cufftDestroy(fwd);
    return MG_ECUDA;
  }
  mg_status st = MG_OK;
  const double ntot = (double)N[0] * N[1] * N[2];
  const long long spec = (long long)N[0] * N[1] * (N[2] / 2 + 1);
  if (cufftSetStream(fwd, s) != CUFFT_SUCCESS || cufftSetStream(inv, s) != CUFFT_SUCCESS ||
      cufftExecD2Z(fwd, R, F) != CUFFT_SUCCESS) {
    st = MG_ECUDA;
  } else {
    k_apply_amplitude<<<grid_for(spec), 256, 0, s>>>(F, N[0], N[1], N[2], h, amp, nt, dk,
                                                     1.0 / (ntot * h * sqrt(h)));
    if (cudaGetLastError() != cudaSuccess || cufftExecZ2D(inv, F, R) != CUFFT_SUCCESS)
      st = MG_ECUDA;
  }
  // the plans' work areas may be released only after their transforms ran
  if (cudaStreamSynchronize(s) != cudaSuccess) st = MG_ECUDA;
  cufftDestroy(fwd);
  cufftDestroy(inv);
  return st;
}

}  // namespace

struct mg_field {
  int n[3] = {0, 0, 0};
  double h = 0.0, dk = 0.0;
  int nt = 0;
  double* amp = nullptr;             // device copy of the table
  cufftDoubleComplex* F = nullptr;   // half spectrum
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  std::string err;
};

extern "C" {

mg_status mg_white_noise(unsigned long long seed, long long n, double* out, void* cuda_stream) {
  if (n < 0 || (n > 0 && !out)) return MG_EINVAL;
  if (n == 0) return MG_OK;
  if (reinterpret_cast<uintptr_t>(out) & 15) return MG_EINVAL;
  k_white_noise<<<grid_for((n + 1) / 2), 256, 0, (cudaStream_t)cuda_stream>>>(seed, 0u, n, out);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ECUDA;
}

mg_status mg_field_create(int n0, int n1, int n2, double h, const double* amp, int nt, double dk,
                          mg_field** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (n0 < 2 || n1 < 2 || n2 < 2 || n0 > 4096 || n1 > 4096 || n2 > 4096 || !(h > 0.0) ||
      !std::isfinite(h) || !amp || nt < 2 || !(dk > 0.0) || !std::isfinite(dk))
    return MG_EINVAL;
  for (int t = 0; t < nt; ++t)
    if (!std::isfinite(amp[t])) return MG_EINVAL;
  mg_field* g = new mg_field();
  g->n[0] = n0;
  g->n[1] = n1;
  g->n[2] = n2;
  g->h = h;
  g->dk = dk;
  g->nt = nt;
  const size_t nspec = (size_t)n0 * n1 * (n2 / 2 + 1);
  mg_status st = MG_OK;
  if (cudaMalloc(&g->amp, nt * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&g->F, nspec * sizeof(cufftDoubleComplex)) != cudaSuccess) {
    st = MG_ENOMEM;
  } else if (cudaMemcpy(g->amp, amp, nt * sizeof(double), cudaMemcpyHostToDevice) !=
             cudaSuccess) {
    st = MG_ECUDA;
  } else if (cufftPlan3d(&g->fwd, n0, n1, n2, CUFFT_D2Z) != CUFFT_SUCCESS) {
    st = MG_ECUDA;
  } else {
    g->have_fwd = true;
    if (cufftPlan3d(&g->inv, n0, n1, n2, CUFFT_Z2D) != CUFFT_SUCCESS)
      st = MG_ECUDA;
    else
      g->have_inv = true;
  }
  if (st != MG_OK) {
    mg_field_destroy(g);
    return st;
  }
  *out = g;
  return MG_OK;
}

mg_status mg_field_convolve(mg_field* g, const double* noise, double* delta, void* cuda_stream) {
  if (!g || !noise || !delta) return MG_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cufftSetStream(g->fwd, s) != CUFFT_SUCCESS || cufftSetStream(g->inv, s) != CUFFT_SUCCESS) {
    g->err = "cufftSetStream failed";
    return MG_ECUDA;
  }
  if (cufftExecD2Z(g->fwd, const_cast<double*>(noise), g->F) != CUFFT_SUCCESS) {
    g->err = "forward transform failed";
    return MG_ECUDA;
  }
  const long long total = (long long)g->n[0] * g->n[1] * (g->n[2] / 2 + 1);
  const double scale = 1.0 / ((double)g->n[0] * g->n[1] * g->n[2]);
  k_apply_amplitude<<<grid_for(total), 256, 0, s>>>(g->F, g->n[0], g->n[1], g->n[2], g->h,
                                                     g->amp, g->nt, g->dk, scale);
  if (cudaGetLastError() != cudaSuccess) {
    g->err = "amplitude kernel launch failed";
    return MG_ECUDA;
  }
  if (cufftExecZ2D(g->inv, g->F, delta) != CUFFT_SUCCESS) {
    g->err = "inverse transform failed";
    return MG_ECUDA;
  }
  return MG_OK;
}

mg_status mg_field_generate(mg_field* g, unsigned long long seed, double* delta,
                            void* cuda_stream) {
  if (!g || !delta) return MG_EINVAL;
  const long long n = (long long)g->n[0] * g->n[1] * g->n[2];
  const mg_status st = mg_white_noise(seed, n, delta, cuda_stream);
  if (st != MG_OK) {
    g->err = "white noise launch failed";
    return st;
  }
  return mg_field_convolve(g, delta, delta, cuda_stream);
}

const char* mg_field_last_error(const mg_field* g) { return g ? g->err.c_str() : ""; }

mg_status mg_density_multiscale(const mg_config* cfg, unsigned long long seed, const double* sqrt_p,
                                int nt, double dk, double* const delta[], void* cuda_stream) {
  if (!cfg || !sqrt_p || nt < 2 || !(dk > 0.0) || !std::isfinite(dk) || !delta) return MG_EINVAL;
  if (mg_config_validate(cfg, nullptr, 0) != MG_OK) return MG_EINVAL;
  for (int t = 0; t < nt; ++t)
    if (!std::isfinite(sqrt_p[t])) return MG_EINVAL;
  const int L = cfg->n_levels;
  for (int l = 0; l < L; ++l)
    if (!delta[l]) return MG_EINVAL;
  int n[MG_MAX_LEVELS][3];
  int off[MG_MAX_LEVELS][3];
  double h[MG_MAX_LEVELS];
  for (int a = 0; a < 3; ++a) n[0][a] = cfg->base_n[a];
  h[0] = cfg->box / cfg->base_n[0];
  size_t max_cells = 0, max_ext = 0, max_real = 0;
  for (int l = 0; l < L; ++l) {
    if (l > 0)
      for (int a = 0; a < 3; ++a) {
        n[l][a] = cfg->nest_n[l - 1][a];
        off[l][a] = cfg->nest_off[l - 1][a];
      }
    if (l > 0) h[l] = h[l - 1] / 2.0;
    const size_t cells = (size_t)n[l][0] * n[l][1] * n[l][2];
    if (cells > max_cells) max_cells = cells;
    if (l < L - 1 && cells > max_ext) max_ext = cells;
    const size_t real = l == 0 ? cells : cells * 8;
    if (real > max_real) max_real = real;
  }
  size_t max_spec = 0;
  for (int l = 0; l < L; ++l) {
    const int f = l == 0 ? 1 : 2;
    const size_t spec = (size_t)f * n[l][0] * f * n[l][1] * (f * n[l][2] / 2 + 1);
    if (spec > max_spec) max_spec = spec;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double *amp = nullptr, *Mprev = nullptr, *Mcur = nullptr, *E = nullptr, *C = nullptr, *R = nullptr;
  cufftDoubleComplex* F = nullptr;
  mg_status st = MG_OK;
  if (cudaMalloc(&amp, nt * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Mprev, max_cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Mcur, max_cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&E, (max_ext ? max_ext : 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&C, max_cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&R, max_real * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&F, max_spec * sizeof(cufftDoubleComplex)) != cudaSuccess)
    st = MG_ENOMEM;
  if (st == MG_OK &&
      cudaMemcpyAsync(amp, sqrt_p, nt * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = MG_ECUDA;
  auto cells_of = [&](int l) { return (long long)n[l][0] * n[l][1] * n[l][2]; };
  auto launched = [&]() { return cudaGetLastError() == cudaSuccess; };
  // base: periodic field of its noise; the field of the noise outside nest 1
  if (st == MG_OK) {
    k_white_noise<<<grid_for((cells_of(0) + 1) / 2), 256, 0, s>>>(seed, 0u, cells_of(0), Mprev);
    k_mask_pad<<<grid_for(cells_of(0)), 256, 0, s>>>(Mprev, n[0][0], n[0][1], n[0][2], R, n[0][0],
                                                     n[0][1], n[0][2], 0, 0, 0, 0, 0, 0);
    if (!launched()) st = MG_ECUDA;
  }
  if (st == MG_OK) st = convolve_grid(n[0], h[0], amp, nt, dk, R, F, s);
  if (st == MG_OK) {
    k_crop<<<grid_for(cells_of(0)), 256, 0, s>>>(R, n[0][1], n[0][2], delta[0], n[0][0], n[0][1],
                                                 n[0][2], nullptr);
    if (L > 1)
      k_mask_pad<<<grid_for(cells_of(0)), 256, 0, s>>>(
          Mprev, n[0][0], n[0][1], n[0][2], R, n[0][0], n[0][1], n[0][2], off[1][0], off[1][1],
          off[1][2], off[1][0] + n[1][0] / 2, off[1][1] + n[1][1] / 2, off[1][2] + n[1][2] / 2);
    if (!launched()) st = MG_ECUDA;
  }
  if (st == MG_OK && L > 1) {
    st = convolve_grid(n[0], h[0], amp, nt, dk, R, F, s);
    if (st == MG_OK) {
      k_crop<<<grid_for(cells_of(0)), 256, 0, s>>>(R, n[0][1], n[0][2], E, n[0][0], n[0][1],
                                                   n[0][2], nullptr);
      if (!launched()) st = MG_ECUDA;
    }
  }
  // nests: constrained noise, isolated field of the own noise + the carried outside field
  for (int l = 1; l < L && st == MG_OK; ++l) {
    const int* m = n[l];
    const int* p = n[l - 1];
    const int N[3] = {2 * m[0], 2 * m[1], 2 * m[2]};
    const long long parents = cells_of(l) / 8;
    k_white_noise<<<grid_for((cells_of(l) + 1) / 2), 256, 0, s>>>(seed, (unsigned)l, cells_of(l),
                                                                    Mcur);
    k_hoffman_ribak<<<grid_for(parents), 256, 0, s>>>(Mcur, m[0], m[1], m[2], Mprev, p[1], p[2],
                                                      off[l][0], off[l][1], off[l][2]);
    k_tricubic<<<grid_for(parents), 128, 0, s>>>(E, p[1], p[2], off[l][0], off[l][1], off[l][2], C,
                                                 m[0], m[1], m[2]);
    k_mask_pad<<<grid_for((long long)N[0] * N[1] * N[2]), 256, 0, s>>>(
        Mcur, m[0], m[1], m[2], R, N[0], N[1], N[2], 0, 0, 0, 0, 0, 0);
    if (!launched()) {
      st = MG_ECUDA;
      break;
    }
    st = convolve_grid(N, h[l], amp, nt, dk, R, F, s);
    if (st != MG_OK) break;
    k_crop<<<grid_for(cells_of(l)), 256, 0, s>>>(R, N[1], N[2], delta[l], m[0], m[1], m[2], C);
    if (l < L - 1) {
      k_mask_pad<<<grid_for((long long)N[0] * N[1] * N[2]), 256, 0, s>>>(
          Mcur, m[0], m[1], m[2], R, N[0], N[1], N[2], off[l + 1][0], off[l + 1][1],
          off[l + 1][2], off[l + 1][0] + n[l + 1][0] / 2, off[l + 1][1] + n[l + 1][1] / 2,
          off[l + 1][2] + n[l + 1][2] / 2);
      if (!launched()) {
        st = MG_ECUDA;
        break;
      }
      st = convolve_grid(N, h[l], amp, nt, dk, R, F, s);
      if (st != MG_OK) break;
      k_crop<<<grid_for(cells_of(l)), 256, 0, s>>>(R, N[1], N[2], E, m[0], m[1], m[2], C);
    }
    if (!launched()) {
      st = MG_ECUDA;
      break;
    }
    double* t = Mprev;
    Mprev = Mcur;
    Mcur = t;
  }
  // covered cells hold the mean of their children, finest first
  for (int l = L - 1; l >= 1 && st == MG_OK; --l) {
    k_children_mean_into<<<grid_for(cells_of(l) / 8), 256, 0, s>>>(
        delta[l], n[l][0], n[l][1], n[l][2], delta[l - 1], n[l - 1][1], n[l - 1][2], off[l][0],
        off[l][1], off[l][2]);
    if (!launched()) st = MG_ECUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && st == MG_OK) st = MG_ECUDA;
  cudaFree(amp);
  cudaFree(Mprev);
  cudaFree(Mcur);
  cudaFree(E);
  cudaFree(C);
  cudaFree(R);
  cudaFree(F);
  return st;
}

mg_status mg_field_destroy(mg_field* g) {
  if (!g) return MG_OK;
  if (g->have_fwd) cufftDestroy(g->fwd);
  if (g->have_inv) cufftDestroy(g->inv);
  cudaFree(g->F);
  cudaFree(g->amp);
  delete g;
  return MG_OK;
}

}  // extern "C"
