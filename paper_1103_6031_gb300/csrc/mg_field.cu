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

// One Philox call per pair of elements; grid-stride over pairs.
__global__ void __launch_bounds__(256)
    k_white_noise(unsigned long long seed, long long n, double* __restrict__ out) {
  const long long pairs = (n + 1) / 2;
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < pairs;
       q += (long long)gridDim.x * blockDim.x) {
    uint32_t x[4] = {(uint32_t)((unsigned long long)q & 0xFFFFFFFFull),
                     (uint32_t)((unsigned long long)q >> 32), 0u, 0u};
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
  k_white_noise<<<grid_for((n + 1) / 2), 256, 0, (cudaStream_t)cuda_stream>>>(seed, n, out);
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
