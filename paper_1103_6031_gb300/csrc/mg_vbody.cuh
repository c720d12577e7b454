// Bodies of the kernels of one float32/float64 V-cycle (Hahn & Abel 2011, Sec. 3.2
// steps 2-9; Sec. 3.3), written once and run two ways: by their own stream kernels
// (one launch per level operation, block and thread indices from the hardware) and
// by the persistent batch kernel (mg_persist.cu), which runs any block of any level
// operation of any hierarchy as a work item of a 128-thread block.  Every body gets
// its block and thread indices as arguments and loads through a policy (Ldg in the
// stream kernels, Weak in the persistent kernel); the arithmetic is the same code,
// so both ways give bit-identical results.
#pragma once

#include "mg_internal.h"
#include "mg_stencil.cuh"

namespace mgk {

// Block and thread indices of one block of a level operation.
struct Blk {
  int bx, by, bz;
  int tx, ty;
};

// Threads along z per block of the smoother and the transfer operations.
constexpr int kVPairX = 32;

// ---- smoother: one colour of red-black Gauss-Seidel, colour-Jacobi ----------------
// Every cell of colour c takes the value that solves its own row of L u = f with all
// other values fixed at their pre-half-sweep values.  Reads uin, writes every interior
// cell of uout (colour c updated, the other colour copied), one z-pair per thread;
// blocks of kVPairX x rows threads.
template <int ORDER, typename T, typename LD>
__device__ __forceinline__ void smooth_half_body(const Grid& G, const T* __restrict__ uin,
                                                 T* __restrict__ uout, const T* __restrict__ f,
                                                 T a_f, int colour, int periodic, int rows, Blk b) {
  const int t = b.bx * kVPairX + b.tx;
  const int j = b.by * rows + b.ty;
  const int i = b.bz;
  const int k0 = 2 * t;
  if (j >= G.n1 || k0 >= G.n2) return;
  const long long sy = G.Zp;
  const long long sx = (long long)G.Y * G.Zp;
  const long long p0 = gidx(G, i, j, k0);
  const int upd = (((i + j + k0) & 1) == colour) ? 0 : 1;
  const bool pair = (k0 + 1) < G.n2;
  if (!pair && upd == 1) {
    const T c = LD::ld(uin + p0);
    uout[p0] = c;
    if (periodic) write_images<T>(G, uout, i, j, k0, c);
    return;
  }
  const long long p = p0 + upd;
  T s1, s2, s3;
  neighbour_sums<ORDER, T, LD>(uin, p, sy, sx, s1, s2, s3);
  // u = (h^2 f - sum_off w u_nb) / w_centre
  constexpr double wc = 3.0 * Lap<ORDER>::w0;
  T v = a_f * LD::ld(f + p);
  v = fma(T(-Lap<ORDER>::w1 / wc), s1, v);
  if (ORDER >= 4) v = fma(T(-Lap<ORDER>::w2 / wc), s2, v);
  if (ORDER >= 6) v = fma(T(-Lap<ORDER>::w3 / wc), s3, v);
  if (pair) {
    typedef typename Vec2<T>::type V2;
    V2 out;
    if (upd == 0) {
      out.x = v;
      out.y = LD::ld(uin + p0 + 1);
    } else {
      out.x = LD::ld(uin + p0);
      out.y = v;
    }
    *reinterpret_cast<V2*>(uout + p0) = out;
    if (periodic) write_pair_images<T>(G, uout, i, j, k0, out.x, out.y);
  } else {
    uout[p0] = v;
    if (periodic) write_images<T>(G, uout, i, j, k0, v);
  }
}

// ---- residual + restriction: one thread per covered parent cell ---------------------
// r = f - L u at its 8 children; parent u := mean(u), ubar := mean(u), parent
// f_fas := mean(r) (L ubar is added by fas_source).  Blocks of 32 x 4 threads.
template <int ORDER, typename T, typename LD>
__device__ __forceinline__ void residual_restrict_body(const Grid& F, const T* __restrict__ u,
                                                       const T* __restrict__ f, T invh2,
                                                       const Grid& P, T* __restrict__ pu,
                                                       T* __restrict__ pfas, T* __restrict__ ubar,
                                                       Int3 off, Int3 cn, int parent_periodic,
                                                       Blk b) {
  const int kc = b.bx * 32 + b.tx;
  const int jc = b.by * 4 + b.ty;
  const int ic = b.bz;
  if (kc >= cn.z || jc >= cn.y) return;
  const long long sy = F.Zp;
  const long long sx = (long long)F.Y * F.Zp;
  T su = T(0), sr = T(0);
#pragma unroll
  for (int di = 0; di < 2; ++di) {
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
#pragma unroll
      for (int dk = 0; dk < 2; ++dk) {
        const long long p = gidx(F, 2 * ic + di, 2 * jc + dj, 2 * kc + dk);
        const T lu = lap_h2<ORDER, T, LD>(u, p, sy, sx);
        su += LD::ld(u + p);
        sr += fma(-invh2, lu, LD::ld(f + p));
      }
    }
  }
  const long long q = gidx(P, off.x + ic, off.y + jc, off.z + kc);
  const T mu = su * T(0.125);
  pu[q] = mu;
  if (parent_periodic) write_images<T>(P, pu, off.x + ic, off.y + jc, off.z + kc, mu);
  pfas[q] = sr * T(0.125);
  ubar[((long long)ic * cn.y + jc) * cn.z + kc] = mu;
}

// ---- FAS source: covered parent cells f_fas += L u (u = restricted fine solution) ----
template <int ORDER, typename T, typename LD>
__device__ __forceinline__ void fas_source_body(const Grid& P, const T* __restrict__ pu,
                                                T* __restrict__ pfas, T invH2, Int3 off, Int3 cn,
                                                Blk b) {
  const int kc = b.bx * 32 + b.tx;
  const int jc = b.by * 4 + b.ty;
  const int ic = b.bz;
  if (kc >= cn.z || jc >= cn.y) return;
  const long long sy = P.Zp;
  const long long sx = (long long)P.Y * P.Zp;
  const long long q = gidx(P, off.x + ic, off.y + jc, off.z + kc);
  pfas[q] = fma(invH2, lap_h2<ORDER, T, LD>(pu, q, sy, sx), pfas[q]);
}

// ---- prolongation-correction: u += inject(parent u - ubar), one thread per z-pair ----
template <typename T, typename LD>
__device__ __forceinline__ void prolong_body(const Grid& F, T* __restrict__ u, const Grid& P,
                                             const T* __restrict__ pu, const T* __restrict__ ubar,
                                             Int3 off, Int3 cn, int periodic, Blk b) {
  const int t = b.bx * 32 + b.tx;
  const int j = b.by * 4 + b.ty;
  const int i = b.bz;
  const int k0 = 2 * t;
  if (j >= F.n1 || k0 >= F.n2) return;
  const int ic = i >> 1, jc = j >> 1, kc = t;
  const T d = LD::ld(pu + gidx(P, off.x + ic, off.y + jc, off.z + kc)) -
              LD::ld(ubar + ((long long)ic * cn.y + jc) * cn.z + kc);
  const long long p = gidx(F, i, j, k0);
  typedef typename Vec2<T>::type V2;
  V2 v = *reinterpret_cast<const V2*>(u + p);
  v.x += d;
  v.y += d;
  *reinterpret_cast<V2*>(u + p) = v;
  if (periodic) {
    if (k0 + 1 < F.n2) write_pair_images<T>(F, u, i, j, k0, v.x, v.y);
    else write_images<T>(F, u, i, j, k0, v.x);
  }
}

// ---- periodic ghost shell: element t of the shell takes its interior image ----------
// (ghost_shell_count(G) elements, mg_internal.h)

template <typename T>
__device__ __forceinline__ void ghost_periodic_body(const Grid& G, T* __restrict__ u, long long t) {
  const long long g = G.g;
  const long long X = G.n0 + 2 * g, Y = G.n1 + 2 * g;
  const long long cntA = X * Y * 2 * g;
  const long long cntB = X * 2 * g * G.n2;
  const long long cntC = 2 * g * (long long)G.n1 * G.n2;
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

// ---- coarse-fine ghosts (Sec. 3.3) ---------------------------------------------------
// The interpolation and flux weights in the kernels' own precision.  The host rounds
// the float64 weights once (round to nearest, the rounding of the device's T(double)
// conversion), so results are bit-identical to converting each weight on the device,
// without the per-use conversions (double-to-float conversions issue on the FP64 pipe,
// which bounded the float32 ghost kernels).
template <typename T>
struct CfW {
  T tang[2][7];
  T ncoarse[3][3];
  T nfine[3][4];
  T flux[6];
};

template <typename T>
inline CfW<T> cf_weights_as(const CfWeights& w) {
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

// Tangential interpolation: thread t handles one parent face element (jc, kc) of a
// layer m: the 4 fine positions over it (tj = 2 jc + pj, tk = 2 kc + pk) interpolate
// the same (n+1) x (n+1) patch of parent values, so each row of the patch is reduced
// along c once per parity pk, then along b once per parity pj.
template <int ORDER, typename T, typename LD>
__device__ __forceinline__ void cf_tangential_body(const Grid& F, const Grid& P,
                                                   const T* __restrict__ pu, Int3 off,
                                                   const FaceSet& fs, const CfW<T>& w, T invH,
                                                   T* __restrict__ inter, T* __restrict__ fc_unc,
                                                   long long t) {
  constexpr int half = ORDER / 2;
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
      const T v = LD::ld(pu + p0 + bb * sb + cc * sc);
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
    for (int s = s0; s < s1; ++s) fc = fma(w.flux[s], LD::ld(pu + q0 + s * sa), fc);
    fc_unc[fs.ebase[f] + (long long)jc * ne1 + kc] = fc * invH;
  }
}

// Normal interpolation and flux matching: thread t handles one fine column of a face;
// the 4 columns under one parent face element are 4 consecutive lanes (a "quad"), which
// share the parent flux and the mean of their fine fluxes through warp shuffles.  Scale
// factors come precomputed: fc_scale = 1/(8 H) for the covered parent cells (mean of 8
// children, parent spacing H); the ghost shift (F_c - mean F_f) h / c_side is
// a_side F_c - b_side (sum of the 4 unscaled fine flux stencils), a_side = h / c_side,
// b_side = 1 / (4 c_side) (c_side: the sum of the flux weights on the ghost side).
// Reads and writes u with plain accesses (the ghosts it writes are not read by it).
template <int ORDER, typename T>
__device__ __forceinline__ void cf_flux_body(const Grid& F, T* __restrict__ u, const FaceSet& fs,
                                             const CfW<T>& w, const T* __restrict__ inter,
                                             const T* __restrict__ fc_unc, T fc_scale, T a0, T a1,
                                             T b0, T b1, int flux_fix, long long t) {
  constexpr int half = ORDER / 2;
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

// ---- coarsest level: periodic pseudo-inverse of L as a circular convolution --------
// u(x) = sum_y K(x - y) f(y), K precomputed on the host from the DFT symbol; block x
// computes output cell x, its kCoarseThreads threads split the sum over y (float64
// sums for either precision); the result also goes to the cell's periodic images.
// Every thread of the block must call it (block-wide reduction).
constexpr int kCoarseThreads = 128;

template <typename T, typename LD>
__device__ __forceinline__ void coarsest_body(const Grid& G, const T* __restrict__ f,
                                              T* __restrict__ u, const double* __restrict__ kern,
                                              int x, int tid) {
  const int n12 = G.n1 * G.n2;
  const int n = G.n0 * n12;
  const int xk = x % G.n2, xj = (x / G.n2) % G.n1, xi = x / n12;
  double acc = 0.0;
  for (int y = tid; y < n; y += kCoarseThreads) {
    const int yk = y % G.n2, yj = (y / G.n2) % G.n1, yi = y / n12;
    int di = xi - yi, dj = xj - yj, dk = xk - yk;
    di += di < 0 ? G.n0 : 0;
    dj += dj < 0 ? G.n1 : 0;
    dk += dk < 0 ? G.n2 : 0;
    acc = fma(__ldg(kern + (di * G.n1 + dj) * G.n2 + dk), (double)LD::ld(f + gidx(G, yi, yj, yk)), acc);
  }
  __shared__ double red[kCoarseThreads];
  red[tid] = acc;
  __syncthreads();
#pragma unroll
  for (int w = kCoarseThreads / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    const T v = (T)red[0];
    u[gidx(G, xi, xj, xk)] = v;
    write_images<T>(G, u, xi, xj, xk, v);
  }
  __syncthreads();  // red[] may be reused by the caller's next block
}

}  // namespace mgk
