// Finite-difference Laplacian of Table 1 (Hahn & Abel 2011, Sec. 3.2): the 3D
// operator is the sum over x, y, z of the 1D second difference of order n,
// i.e. 7, 13 or 19 points.  Weights below are the 1D weights on offsets
// 0, +-1, +-2, +-3 (units 1/h^2).
#pragma once

#include "mg_internal.h"

namespace mgk {

template <int ORDER>
struct Lap;
template <>
struct Lap<2> {
  static constexpr double w0 = -2.0, w1 = 1.0, w2 = 0.0, w3 = 0.0;
};
template <>
struct Lap<4> {
  static constexpr double w0 = -30.0 / 12.0, w1 = 16.0 / 12.0, w2 = -1.0 / 12.0, w3 = 0.0;
};
template <>
struct Lap<6> {
  static constexpr double w0 = -490.0 / 180.0, w1 = 270.0 / 180.0, w2 = -27.0 / 180.0,
                          w3 = 2.0 / 180.0;
};

// Sums of the 6 neighbours at distance d = 1, 2, 3 (axis-aligned) of element p.
template <int ORDER, typename T>
__device__ __forceinline__ void neighbour_sums(const T* __restrict__ u, long long p, long long sy,
                                               long long sx, T& s1, T& s2, T& s3) {
  s1 = (__ldg(u + p - 1) + __ldg(u + p + 1)) + (__ldg(u + p - sy) + __ldg(u + p + sy)) +
       (__ldg(u + p - sx) + __ldg(u + p + sx));
  s2 = T(0);
  s3 = T(0);
  if (ORDER >= 4) {
    s2 = (__ldg(u + p - 2) + __ldg(u + p + 2)) + (__ldg(u + p - 2 * sy) + __ldg(u + p + 2 * sy)) +
         (__ldg(u + p - 2 * sx) + __ldg(u + p + 2 * sx));
  }
  if (ORDER >= 6) {
    s3 = (__ldg(u + p - 3) + __ldg(u + p + 3)) + (__ldg(u + p - 3 * sy) + __ldg(u + p + 3 * sy)) +
         (__ldg(u + p - 3 * sx) + __ldg(u + p + 3 * sx));
  }
}

// h^2 L u at element p.
template <int ORDER, typename T>
__device__ __forceinline__ T lap_h2(const T* __restrict__ u, long long p, long long sy,
                                    long long sx) {
  T s1, s2, s3;
  neighbour_sums<ORDER, T>(u, p, sy, sx, s1, s2, s3);
  T acc = T(3.0 * Lap<ORDER>::w0) * __ldg(u + p);
  acc = fma(T(Lap<ORDER>::w1), s1, acc);
  if (ORDER >= 4) acc = fma(T(Lap<ORDER>::w2), s2, acc);
  if (ORDER >= 6) acc = fma(T(Lap<ORDER>::w3), s3, acc);
  return acc;
}

// On a periodic level, every ghost cell is the image of one interior cell (all
// sides are >= g).  Writes v to the images of interior cell (i, j, k); the cell
// itself is written by the caller.
template <typename T>
__device__ __forceinline__ void write_images(const Grid& G, T* __restrict__ u, int i, int j,
                                             int k, T v) {
  const int g = G.g;
  if (i >= g && i < G.n0 - g && j >= g && j < G.n1 - g && k >= g && k < G.n2 - g) return;
  int is[2], js[2], ks[2];
  int ni = 0, nj = 0, nk = 0;
  if (i < g) is[ni++] = i + G.n0;
  if (i >= G.n0 - g) is[ni++] = i - G.n0;
  if (j < g) js[nj++] = j + G.n1;
  if (j >= G.n1 - g) js[nj++] = j - G.n1;
  if (k < g) ks[nk++] = k + G.n2;
  if (k >= G.n2 - g) ks[nk++] = k - G.n2;
  // all combinations of (own or image) per axis, except own on every axis
  for (int a = 0; a <= ni; ++a)
    for (int b = 0; b <= nj; ++b)
      for (int c = 0; c <= nk; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        const int ii = a == 0 ? i : is[a - 1];
        const int jj = b == 0 ? j : js[b - 1];
        const int kk = c == 0 ? k : ks[c - 1];
        u[gidx(G, ii, jj, kk)] = v;
      }
}

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  typedef double2 type;
};
template <>
struct Vec2<float> {
  typedef float2 type;
};

}  // namespace mgk
