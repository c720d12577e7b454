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

// Load policies.  Ldg: the read-only data path, for kernels whose inputs no thread of
// the launch writes.  Weak: plain loads, for the persistent kernel, whose work items
// read what earlier items of the same launch wrote (ordered by release/acquire
// flags, which the read-only path does not observe).
struct Ldg {
  template <typename T>
  static __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }
};
struct Weak {
  template <typename T>
  static __device__ __forceinline__ T ld(const T* p) { return *p; }
};

// Sums of the 6 neighbours at distance d = 1, 2, 3 (axis-aligned) of element p.
template <int ORDER, typename T, typename LD = Ldg>
__device__ __forceinline__ void neighbour_sums(const T* __restrict__ u, long long p, long long sy,
                                               long long sx, T& s1, T& s2, T& s3) {
  s1 = (LD::ld(u + p - 1) + LD::ld(u + p + 1)) + (LD::ld(u + p - sy) + LD::ld(u + p + sy)) +
       (LD::ld(u + p - sx) + LD::ld(u + p + sx));
  s2 = T(0);
  s3 = T(0);
  if (ORDER >= 4) {
    s2 = (LD::ld(u + p - 2) + LD::ld(u + p + 2)) + (LD::ld(u + p - 2 * sy) + LD::ld(u + p + 2 * sy)) +
         (LD::ld(u + p - 2 * sx) + LD::ld(u + p + 2 * sx));
  }
  if (ORDER >= 6) {
    s3 = (LD::ld(u + p - 3) + LD::ld(u + p + 3)) + (LD::ld(u + p - 3 * sy) + LD::ld(u + p + 3 * sy)) +
         (LD::ld(u + p - 3 * sx) + LD::ld(u + p + 3 * sx));
  }
}

// h^2 L u at element p.
template <int ORDER, typename T, typename LD = Ldg>
__device__ __forceinline__ T lap_h2(const T* __restrict__ u, long long p, long long sy,
                                    long long sx) {
  T s1, s2, s3;
  neighbour_sums<ORDER, T, LD>(u, p, sy, sx, s1, s2, s3);
  T acc = T(3.0 * Lap<ORDER>::w0) * LD::ld(u + p);
  acc = fma(T(Lap<ORDER>::w1), s1, acc);
  if (ORDER >= 4) acc = fma(T(Lap<ORDER>::w2), s2, acc);
  if (ORDER >= 6) acc = fma(T(Lap<ORDER>::w3), s3, acc);
  return acc;
}

// On a periodic level, every ghost cell is the image of one interior cell (all
// sides are >= g).  Along an axis of n cells with element stride st, index a has
// an image at a + n when a < g and at a - n when a >= n - g (both when n < 2g);
// ImgAxis holds the element offsets of those images, 0 for none.
struct ImgAxis {
  long long lo, hi;
};

__device__ __forceinline__ ImgAxis img_axis(int a, int n, int g, long long st) {
  return ImgAxis{a < g ? (long long)n * st : 0, a >= n - g ? -(long long)n * st : 0};
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

// Writes v to the images of interior cell (i, j, k): every combination of own
// or image index per axis except own on every axis.  Straight-line predicated
// stores (the loops unroll; no local memory); the cell itself is written by the
// caller.
template <typename T>
__device__ __forceinline__ void write_images(const Grid& G, T* __restrict__ u, int i, int j,
                                             int k, T v) {
  const int g = G.g;
  if (i >= g && i < G.n0 - g && j >= g && j < G.n1 - g && k >= g && k < G.n2 - g) return;
  const long long sy = G.Zp, sx = (long long)G.Y * G.Zp;
  const ImgAxis ax = img_axis(i, G.n0, g, sx), ay = img_axis(j, G.n1, g, sy),
                az = img_axis(k, G.n2, g, 1);
  T* p = u + gidx(G, i, j, k);
  const long long ox[3] = {0, ax.lo, ax.hi}, oy[3] = {0, ay.lo, ay.hi}, oz[3] = {0, az.lo, az.hi};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if ((a | b | c) && (a == 0 || ox[a]) && (b == 0 || oy[b]) && (c == 0 || oz[c]))
          p[ox[a] + oy[b] + oz[c]] = v;
}

// Images of the z-pair (k, k+1), k even and k + 1 < n2, with values (va, vb): the
// x/y images of the pair as one vector store each (x and y offsets are multiples
// of the row pitch, so the alignment of the pair is kept), the z images of each
// cell scalar, at the cell's own row and at every x/y image row.
template <typename T>
__device__ __forceinline__ void write_pair_images(const Grid& G, T* __restrict__ u, int i, int j,
                                                  int k, T va, T vb) {
  const int g = G.g;
  if (i >= g && i < G.n0 - g && j >= g && j < G.n1 - g && k >= g && k + 1 < G.n2 - g) return;
  typedef typename Vec2<T>::type V2;
  const long long sy = G.Zp, sx = (long long)G.Y * G.Zp;
  const ImgAxis ax = img_axis(i, G.n0, g, sx), ay = img_axis(j, G.n1, g, sy);
  const ImgAxis z0 = img_axis(k, G.n2, g, 1), z1 = img_axis(k + 1, G.n2, g, 1);
  T* p = u + gidx(G, i, j, k);
  const long long ox[3] = {0, ax.lo, ax.hi}, oy[3] = {0, ay.lo, ay.hi};
  V2 pv;
  pv.x = va;
  pv.y = vb;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if ((a != 0 && !ox[a]) || (b != 0 && !oy[b])) continue;
      T* q = p + ox[a] + oy[b];
      if (a | b) *reinterpret_cast<V2*>(q) = pv;
      if (z0.lo) q[z0.lo] = va;
      if (z0.hi) q[z0.hi] = va;
      if (z1.lo) q[1 + z1.lo] = vb;
      if (z1.hi) q[1 + z1.hi] = vb;
    }
}

}  // namespace mgk
