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

namespace mgk {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_ghost_periodic(Grid G, T* __restrict__ u) {
  const long long g = G.g;
  const long long X = G.n0 + 2 * g, Y = G.n1 + 2 * g;
  const long long cntA = X * Y * 2 * g;
  const long long cntB = X * 2 * g * G.n2;
  const long long cntC = 2 * g * (long long)G.n1 * G.n2;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int i, j, k;
  if (t < cntA) {
    const int kk = (int)(t % (2 * g));
    t /= 2 * g;
    j = (int)(t % Y) - (int)g;
    i = (int)(t / Y) - (int)g;
    k = kk < g ? kk - (int)g : G.n2 + kk - (int)g;
  } else if (t < cntA + cntB) {
    t -= cntA;
    k = (int)(t % G.n2);
    t /= G.n2;
    const int jj = (int)(t % (2 * g));
    i = (int)(t / (2 * g)) - (int)g;
    j = jj < g ? jj - (int)g : G.n1 + jj - (int)g;
  } else if (t < cntA + cntB + cntC) {
    t -= cntA + cntB;
    k = (int)(t % G.n2);
    t /= G.n2;
    j = (int)(t % G.n1);
    const int ii = (int)(t / G.n1);
    i = ii < g ? ii - (int)g : G.n0 + ii - (int)g;
  } else {
    return;
  }
  const int si = ((i % G.n0) + G.n0) % G.n0;
  const int sj = ((j % G.n1) + G.n1) % G.n1;
  const int sk = ((k % G.n2) + G.n2) % G.n2;
  u[gidx(G, i, j, k)] = u[gidx(G, si, sj, sk)];
}

// The interpolation and flux weights in the kernels' own precision.  The host
// rounds the float64 weights once (round to nearest, the rounding of the device's
// T(double) conversion), so results are bit-identical to converting each weight on
// the device, without the per-use conversions (double to float conversions issue on
// the FP64 pipe, which bounded the float32 ghost kernels).
template <typename T>
struct CfW {
  T tang[2][7];
  T ncoarse[3][3];
  T nfine[3][4];
  T flux[6];
};

template <typename T>
CfW<T> cf_weights_as(const CfWeights& w) {
  CfW<T> o;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 7; ++b) o.tang[a][b] = T(w.tang[a][b]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) o.ncoarse[a][b] = T(w.ncoarse[a][b]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 4; ++b) o.nfine[a][b] = T(w.nfine[a][b]);
  for (int a = 0; a < 6; ++a) o.flux[a] = T(w.flux[a]);
  return o;
}

__device__ __forceinline__ void face_axes(int a, int& b, int& c) {
  b = (a == 0) ? 1 : 0;
  c = (a == 2) ? 1 : 2;
}

__device__ __forceinline__ int face_of(const FaceSet& fs, long long t, const long long* base) {
  int f = 0;
#pragma unroll
  for (int q = 1; q < 6; ++q)
    if (t >= base[q]) f = q;
  return f;
}

// One thread per parent face element (jc, kc) of a layer m: the 4 fine positions
// over it (tj = 2 jc + pj, tk = 2 kc + pk) interpolate the same (n+1) x (n+1)
// patch of parent values, so each row of the patch is reduced along c once per
// parity pk, then along b once per parity pj (each value is the same chain of fmas
// as the per-position form: a quarter of the loads, ~0.56 of the float64 work).
template <int ORDER, typename T>
__global__ void __launch_bounds__(128)
    k_cf_tangential(Grid F, Grid P, const T* __restrict__ pu, Int3 off, FaceSet fs, CfW<T> w,
                    T invH, T* __restrict__ inter, T* __restrict__ fc_unc) {
  constexpr int half = ORDER / 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= half * fs.ebase[6]) return;
  int f = 0;
#pragma unroll
  for (int q = 1; q < 6; ++q)
    if (t >= half * fs.ebase[q]) f = q;
  const int a = f >> 1, side = f & 1;
  int b, c;
  face_axes(a, b, c);
  const int nt0 = fs.nt[f][0], nt1 = fs.nt[f][1];
  const int ne1 = nt1 / 2;
  const long long ne = (long long)(nt0 / 2) * ne1;
  long long loc = t - half * fs.ebase[f];
  const int m = (int)(loc / ne);
  loc -= (long long)m * ne;
  const int jc = (int)(loc / ne1), kc = (int)(loc % ne1);
  auto pick = [](int ax, int x, int y, int z) { return ax == 0 ? x : (ax == 1 ? y : z); };
  const int off_a = pick(a, off.x, off.y, off.z), nf_a = pick(a, F.n0, F.n1, F.n2);
  const int pn = side == 0 ? off_a - 1 - m : off_a + nf_a / 2 + m;
  const int pb = pick(b, off.x, off.y, off.z) + jc, pc = pick(c, off.x, off.y, off.z) + kc;
  // parent element strides along a, b, c and the patch corner (pn, pb - half, pc - half)
  const long long sxP = (long long)P.Y * P.Zp, syP = P.Zp;
  auto stride = [&](int ax) { return ax == 0 ? sxP : (ax == 1 ? syP : 1LL); };
  const long long sa = stride(a), sb = stride(b), sc = stride(c);
  auto coord = [&](int ax, int va, int vb, int vc) { return ax == a ? va : (ax == b ? vb : vc); };
  const long long p0 = gidx(P, coord(0, pn, pb - half, pc - half), coord(1, pn, pb - half, pc - half),
                            coord(2, pn, pb - half, pc - half));
  T row[2][ORDER + 1];
#pragma unroll
  for (int bb = 0; bb <= ORDER; ++bb) {
    T r0 = T(0), r1 = T(0);
#pragma unroll
    for (int cc = 0; cc <= ORDER; ++cc) {
      const T v = __ldg(pu + p0 + bb * sb + cc * sc);
      r0 = fma(w.tang[0][cc], v, r0);
      r1 = fma(w.tang[1][cc], v, r1);
    }
    row[0][bb] = r0;
    row[1][bb] = r1;
  }
  typedef typename Vec2<T>::type V2;
#pragma unroll
  for (int pj = 0; pj < 2; ++pj) {
    T acc0 = T(0), acc1 = T(0);
#pragma unroll
    for (int bb = 0; bb <= ORDER; ++bb) {
      acc0 = fma(w.tang[pj][bb], row[0][bb], acc0);
      acc1 = fma(w.tang[pj][bb], row[1][bb], acc1);
    }
    // (tk, tk + 1) = (2 kc, 2 kc + 1): an even, hence 2-element aligned, pair
    V2 out;
    out.x = acc0;
    out.y = acc1;
    *reinterpret_cast<V2*>(inter + fs.base[f] + ((long long)m * nt0 + 2 * jc + pj) * nt1 + 2 * kc) =
        out;
  }
  if (m == 0) {
    // uncovered part of the parent face flux for element (jc, kc): parent cells
    // pface - half + s along a, s0 <= s < s1, at (pb, pc)
    const int pface = side == 0 ? off_a : off_a + nf_a / 2;
    const long long q0 = p0 + half * sb + half * sc + (long long)(pface - half - pn) * sa;
    T fc = T(0);
    const int s0 = side == 0 ? 0 : half, s1 = side == 0 ? half : ORDER;
    for (int s = s0; s < s1; ++s) fc = fma(w.flux[s], __ldg(pu + q0 + s * sa), fc);
    fc_unc[fs.ebase[f] + (long long)jc * ne1 + kc] = fc * invH;
  }
}

// One thread per fine column of a face; the 4 columns under one parent face
// element are 4 consecutive lanes (a "quad"), which share the parent flux and
// the mean of their fine fluxes through warp shuffles.  Scale factors come
// precomputed (the float64 pipe is this kernel's bound): fc_scale = 1/(8 H) for the
// covered parent cells (mean of 8 children, parent spacing H); the ghost shift
// (F_c - mean F_f) h / c_side is a_side F_c - b_side (sum of the 4 unscaled fine
// flux stencils), a_side = h / c_side, b_side = 1 / (4 c_side) (c_side: the sum of
// the flux weights on the ghost side).
template <int ORDER, typename T>
__global__ void __launch_bounds__(128)
    k_cf_flux(Grid F, T* __restrict__ u, FaceSet fs, CfW<T> w, const T* __restrict__ inter,
              const T* __restrict__ fc_unc, T fc_scale, T a0, T a1, T b0, T b1, int flux_fix) {
  constexpr int half = ORDER / 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 4 * fs.ebase[6]) return;
  const unsigned quad = __activemask();
  const long long e = t >> 2;
  const int col = (int)(t & 3);
  const int f = face_of(fs, e, fs.ebase);
  const int a = f >> 1, side = f & 1;
  const int nt0 = fs.nt[f][0], nt1 = fs.nt[f][1];
  const long long loc = e - fs.ebase[f];
  const int jc = (int)(loc / (nt1 / 2)), kc = (int)(loc % (nt1 / 2));
  const int tj = 2 * jc + (col >> 1), tk = 2 * kc + (col & 1);
  const long long sx = (long long)F.Y * F.Zp, sy = F.Zp;
  // strides along the normal (a) and the tangential axes (b, c) of this face
  const long long sa = a == 0 ? sx : (a == 1 ? sy : 1);
  const long long sb = a == 0 ? sy : sx;
  const long long sc = a == 2 ? sy : 1;
  const int na = a == 0 ? F.n0 : (a == 1 ? F.n1 : F.n2);
  // element (0 along the normal, tj, tk); moving inwards is +sa (low face) or -sa (high)
  const long long col0 = gidx(F, 0, 0, 0) + tj * sb + tk * sc;
  const long long in0 = side == 0 ? col0 : col0 + (long long)(na - 1) * sa;
  const long long step = side == 0 ? sa : -sa;
  // fine interior values q = 0 .. half from the face
  T v[half + 1];
#pragma unroll
  for (int q = 0; q <= half; ++q) v[q] = u[in0 + q * step];
  // parent flux: uncovered part + covered parent cells as the mean of their 8
  // children; each column holds 2 of the 8 (normal 2d, 2d+1)
  T cov = T(0);
#pragma unroll
  for (int d = 0; d < half; ++d) {
    const int s = side == 0 ? half + d : half - 1 - d;
    T pair = u[in0 + (2 * d) * step] + u[in0 + (2 * d + 1) * step];
    pair += __shfl_xor_sync(quad, pair, 1);
    pair += __shfl_xor_sync(quad, pair, 2);
    cov = fma(w.flux[s], pair, cov);
  }
  const T fc = fma(cov, fc_scale, fc_unc[e]);
  T cq[half];
#pragma unroll
  for (int q = 0; q < half; ++q) cq[q] = inter[fs.base[f] + ((long long)q * nt0 + tj) * nt1 + tk];
  T ghost[half];
#pragma unroll
  for (int m = 0; m < half; ++m) {
    T gv = T(0);
#pragma unroll
    for (int q = 0; q < half; ++q) gv = fma(w.ncoarse[m][q], cq[q], gv);
#pragma unroll
    for (int q = 0; q <= half; ++q) gv = fma(w.nfine[m][q], v[q], gv);
    ghost[m] = gv;
  }
  T ff = T(0);
#pragma unroll
  for (int s = 0; s < ORDER; ++s) {
    T x;
    if (side == 0) x = s < half ? ghost[half - 1 - s] : v[s - half];
    else x = s < half ? v[half - 1 - s] : ghost[s - half];
    ff = fma(w.flux[s], x, ff);
  }
  ff += __shfl_xor_sync(quad, ff, 1);
  ff += __shfl_xor_sync(quad, ff, 2);
  T shift = T(0);
  if (flux_fix) shift = fma(-(side ? b1 : b0), ff, fc * (side ? a1 : a0));
#pragma unroll
  for (int m = 0; m < half; ++m) u[in0 - (m + 1) * step] = ghost[m] + shift;
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
