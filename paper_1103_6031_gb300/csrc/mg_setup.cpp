// Host-side set-up that needs no GPU: level geometry, coarse-fine interpolation
// weights (Lagrange form), face-flux weights derived from the Laplacian by
// telescoping, and the periodic pseudo-inverse kernel of the coarsest level.
#include <cmath>
#include <cstring>
#include <vector>

#include "mg_internal.h"
#include "mg_setup.h"

namespace mgk {

Grid make_grid(int n0, int n1, int n2, int g) {
  Grid G;
  G.n0 = n0;
  G.n1 = n1;
  G.n2 = n2;
  G.g = g;
  G.za = 4;
  G.Y = n1 + 2 * g;
  G.X = n0 + 2 * g;
  const int need = G.za + n2 + g;
  G.Zp = (need + 7) / 8 * 8;
  return G;
}

// 1D Laplacian weights of Table 1 on offsets -half..half.
void laplacian_1d(int order, double* w) {
  if (order == 2) {
    const double v[3] = {1.0, -2.0, 1.0};
    std::memcpy(w, v, sizeof(v));
  } else if (order == 4) {
    const double v[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
    for (int i = 0; i < 5; ++i) w[i] = v[i] / 12.0;
  } else {
    const double v[7] = {2.0, -27.0, 270.0, -490.0, 270.0, -27.0, 2.0};
    for (int i = 0; i < 7; ++i) w[i] = v[i] / 180.0;
  }
}

static double lagrange(const double* nodes, int count, int j, double x) {
  double w = 1.0;
  for (int m = 0; m < count; ++m)
    if (m != j) w *= (x - nodes[m]) / (nodes[j] - nodes[m]);
  return w;
}

void compute_cf_weights(int order, CfWeights* w) {
  std::memset(w, 0, sizeof(*w));
  const int half = order / 2;
  // parallel to the face: n+1 parent centres -half..half (parent units), fine
  // centre at -1/4 (even fine index) or +1/4 (odd)
  double tn[7];
  for (int s = 0; s <= order; ++s) tn[s] = s - half;
  for (int p = 0; p < 2; ++p) {
    const double x = p == 0 ? -0.25 : 0.25;
    for (int s = 0; s <= order; ++s) w->tang[p][s] = lagrange(tn, order + 1, s, x);
  }
  // normal to the face (fine units from the face, positive inwards): parent
  // centres at -1, -3, ...; fine centres at 1/2, 3/2, ...; ghosts at -1/2, -3/2, ...
  double nn[7];
  for (int q = 0; q < half; ++q) nn[q] = -(2.0 * q + 1.0);
  for (int q = 0; q <= half; ++q) nn[half + q] = q + 0.5;
  for (int m = 0; m < half; ++m) {
    const double x = -(m + 0.5);
    for (int q = 0; q < half; ++q) w->ncoarse[m][q] = lagrange(nn, order + 1, q, x);
    for (int q = 0; q <= half; ++q) w->nfine[m][q] = lagrange(nn, order + 1, half + q, x);
  }
  // face flux F_{i+1/2} on cells i-half+1 .. i+half with F_{i+1/2} - F_{i-1/2} = L_i:
  // c_m = -(l_0 + ... + l_m)
  double l[7];
  laplacian_1d(order, l);
  double acc = 0.0;
  for (int m = 0; m < order; ++m) {
    acc += l[m];
    w->flux[m] = -acc;
  }
  w->ghost_coef[0] = 0.0;
  w->ghost_coef[1] = 0.0;
  for (int s = 0; s < half; ++s) w->ghost_coef[0] += w->flux[s];
  for (int s = half; s < order; ++s) w->ghost_coef[1] += w->flux[s];
}

void make_faceset(const Grid& F, int half, FaceSet* fs) {
  const int n[3] = {F.n0, F.n1, F.n2};
  fs->base[0] = 0;
  fs->ebase[0] = 0;
  for (int f = 0; f < 6; ++f) {
    const int a = f >> 1;
    const int b = a == 0 ? 1 : 0;
    const int c = a == 2 ? 1 : 2;
    fs->nt[f][0] = n[b];
    fs->nt[f][1] = n[c];
    fs->base[f + 1] = fs->base[f] + (long long)half * n[b] * n[c];
    fs->ebase[f + 1] = fs->ebase[f] + (long long)(n[b] / 2) * (n[c] / 2);
  }
}

// Zero-mean periodic inverse of L on an m0 x m1 x m2 grid of spacing h as a
// convolution kernel: K(d) = (1/M) sum_{k != 0} exp(i k.d) / lambda(k), lambda
// the DFT eigenvalue of L.  lambda is even in every k_a, so the sum is a
// product of cosine transforms along each axis.
void coarsest_kernel(int order, int m0, int m1, int m2, double h, std::vector<double>& K) {
  double l[7];
  laplacian_1d(order, l);
  const int half = order / 2;
  const int m[3] = {m0, m1, m2};
  std::vector<double> lam1[3], cs[3];
  for (int a = 0; a < 3; ++a) {
    lam1[a].resize(m[a]);
    cs[a].resize((size_t)m[a] * m[a]);
    for (int k = 0; k < m[a]; ++k) {
      const double th = 2.0 * M_PI * k / m[a];
      double v = l[half];
      for (int s = 1; s <= half; ++s) v += 2.0 * l[half + s] * std::cos(s * th);
      lam1[a][k] = v / (h * h);
      for (int d = 0; d < m[a]; ++d) cs[a][(size_t)k * m[a] + d] = std::cos(th * d);
    }
  }
  const size_t M = (size_t)m0 * m1 * m2;
  std::vector<double> inv(M);
  for (int k0 = 0; k0 < m0; ++k0)
    for (int k1 = 0; k1 < m1; ++k1)
      for (int k2 = 0; k2 < m2; ++k2) {
        const double lam = lam1[0][k0] + lam1[1][k1] + lam1[2][k2];
        const size_t q = ((size_t)k0 * m1 + k1) * m2 + k2;
        inv[q] = (k0 == 0 && k1 == 0 && k2 == 0) ? 0.0 : 1.0 / lam;
      }
  // transform along z, then y, then x
  std::vector<double> t1(M), t2(M);
  for (int k0 = 0; k0 < m0; ++k0)
    for (int k1 = 0; k1 < m1; ++k1)
      for (int d2 = 0; d2 < m2; ++d2) {
        double s = 0.0;
        for (int k2 = 0; k2 < m2; ++k2)
          s += cs[2][(size_t)k2 * m2 + d2] * inv[((size_t)k0 * m1 + k1) * m2 + k2];
        t1[((size_t)k0 * m1 + k1) * m2 + d2] = s;
      }
  for (int k0 = 0; k0 < m0; ++k0)
    for (int d1 = 0; d1 < m1; ++d1)
      for (int d2 = 0; d2 < m2; ++d2) {
        double s = 0.0;
        for (int k1 = 0; k1 < m1; ++k1)
          s += cs[1][(size_t)k1 * m1 + d1] * t1[((size_t)k0 * m1 + k1) * m2 + d2];
        t2[((size_t)k0 * m1 + d1) * m2 + d2] = s;
      }
  K.assign(M, 0.0);
  for (int d0 = 0; d0 < m0; ++d0)
    for (int d1 = 0; d1 < m1; ++d1)
      for (int d2 = 0; d2 < m2; ++d2) {
        double s = 0.0;
        for (int k0 = 0; k0 < m0; ++k0)
          s += cs[0][(size_t)k0 * m0 + d0] * t2[((size_t)k0 * m1 + d1) * m2 + d2];
        K[((size_t)d0 * m1 + d1) * m2 + d2] = s / (double)M;
      }
}

// Level chain: full coarsenings of the base (coarsest first), base, nests.
bool build_levels(const mg_config* cfg, std::vector<LevelGeom>& out, int* base_index, char* msg,
                  size_t len) {
  out.clear();
  const int order = cfg->order;
  const int g = order / 2;
  std::vector<LevelGeom> chain;
  LevelGeom b;
  b.n[0] = cfg->base_n[0];
  b.n[1] = cfg->base_n[1];
  b.n[2] = cfg->base_n[2];
  b.h = cfg->box / cfg->base_n[0];
  b.nest = false;
  b.off[0] = b.off[1] = b.off[2] = 0;
  chain.push_back(b);
  for (;;) {
    const LevelGeom& c = chain.back();
    const bool even = c.n[0] % 2 == 0 && c.n[1] % 2 == 0 && c.n[2] % 2 == 0;
    int mx = c.n[0], mn = c.n[0];
    for (int a = 1; a < 3; ++a) {
      if (c.n[a] > mx) mx = c.n[a];
      if (c.n[a] < mn) mn = c.n[a];
    }
    if (!(even && mx > 8 && mn / 2 >= g)) break;
    LevelGeom d = c;
    for (int a = 0; a < 3; ++a) d.n[a] = c.n[a] / 2;
    d.h = c.h * 2.0;
    chain.push_back(d);
  }
  for (int i = (int)chain.size() - 1; i >= 0; --i) out.push_back(chain[i]);
  *base_index = (int)chain.size() - 1;
  const LevelGeom& coarsest = out[0];
  const long long cells = (long long)coarsest.n[0] * coarsest.n[1] * coarsest.n[2];
  if (cells > 32768) {
    if (msg && len) snprintf(msg, len, "coarsest level has %lld cells (> 32768); use a base whose sides halve further", cells);
    return false;
  }
  double h = b.h;
  int parent[3] = {b.n[0], b.n[1], b.n[2]};
  for (int i = 0; i + 1 < cfg->n_levels; ++i) {
    LevelGeom nl;
    h *= 0.5;
    nl.h = h;
    nl.nest = true;
    for (int a = 0; a < 3; ++a) {
      nl.n[a] = cfg->nest_n[i][a];
      nl.off[a] = cfg->nest_off[i][a];
      const int min_side = order > 4 ? order : 4;
      if (nl.n[a] < min_side || nl.n[a] % 2 != 0) {
        if (msg && len) snprintf(msg, len, "nest %d: size %d on axis %d must be even and >= %d", i, nl.n[a], a, min_side);
        return false;
      }
      if (nl.off[a] < order || nl.off[a] + nl.n[a] / 2 + order > parent[a]) {
        if (msg && len)
          snprintf(msg, len, "nest %d axis %d: region [%d, %d) of a parent of %d cells leaves less than %d parent cells of margin",
                   i, a, nl.off[a], nl.off[a] + nl.n[a] / 2, parent[a], order);
        return false;
      }
    }
    out.push_back(nl);
    for (int a = 0; a < 3; ++a) parent[a] = nl.n[a];
  }
  return true;
}

}  // namespace mgk
