// Hierarchy object, FAS V-cycle driver and the C ABI of include/mg.h.
//
// The V-cycle follows Hahn & Abel 2011, Sec. 3.2 (enumerated algorithm) on the
// composite grid of Sec. 3.3: levels below the base are full periodic
// coarsenings, the base is periodic, nests take their boundary values from
// the parent through coarse-fine interpolation with flux matching.  Every step
// is a kernel launch on the hierarchy's stream; the host only sequences them
// and reads back one convergence record per cycle.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mg.h"
#include "mg_internal.h"
#include "mg_setup.h"

using namespace mgk;

namespace {

struct DevLevel {
  LevelGeom geo;
  Grid G;
  bool periodic = true;
  bool leaf = false;
  bool has_child = false;
  Int3 off{0, 0, 0};  // origin in parent cells
  Int3 cn{0, 0, 0};   // covered extent in the parent
  Int3 child_lo{0, 0, 0}, child_hi{0, 0, 0};  // region covered by the child, own cells
  double* u[2] = {nullptr, nullptr};
  int cur = 0;
  // Periodic levels: every kernel that writes u also writes its ghost images,
  // so ghosts are refilled only after u is loaded from outside.
  bool ghosts_stale = true;
  double* f = nullptr;
  double* ffas = nullptr;
  double* ubar = nullptr;
  FaceSet fs;
  double* inter = nullptr;
  double* fc_unc = nullptr;
  double* kern = nullptr;
  int nblocks = 0;
  int partial_off = 0;
};

struct Plan {
  std::vector<LevelGeom> geo;
  int base = 0;
  size_t bytes = 0;
};

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

double centre_weight(int order) {
  double l[7];
  laplacian_1d(order, l);
  return 3.0 * l[order / 2];
}

}  // namespace

struct mg_hierarchy {
  mg_config cfg;
  std::vector<DevLevel> L;
  int base = 0;
  cudaStream_t s = nullptr;
  CfWeights w;
  std::string err;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  double* partial = nullptr;
  int partial_slots = 0;
  double* red = nullptr;       // [0..1] norm sums, [2..3] source sum
  double* host_red = nullptr;  // pinned copy of red
  double* scratch = nullptr;   // 3 dense arrays of the largest leaf level
  long long scratch_elems = 0;
  double volume = 0.0;
  // launch counters and optional CUDA-event timing per kernel family
  mg_stats stats;
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> ev_start[MG_K_FAMILIES], ev_end[MG_K_FAMILIES];
  size_t ev_used[MG_K_FAMILIES] = {0};
};

namespace {

mg_status fail(mg_hierarchy* h, mg_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

mg_status fail_cuda(mg_hierarchy* h, cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return fail(h, MG_ECUDA, buf);
}

#define CK(expr)                                                 \
  do {                                                           \
    cudaError_t e_ = (expr);                                     \
    if (e_ != cudaSuccess) return fail_cuda(h, e_, #expr);       \
  } while (0)

#define ST(expr)                       \
  do {                                 \
    mg_status st_ = (expr);            \
    if (st_ != MG_OK) return st_;      \
  } while (0)

mg_status prof_begin(mg_hierarchy* h, int fam) {
  if (!(h->prof_mask & (1u << fam))) return MG_OK;
  size_t& used = h->ev_used[fam];
  if (used == h->ev_start[fam].size()) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    h->ev_start[fam].push_back(a);
    h->ev_end[fam].push_back(b);
  }
  CK(cudaEventRecord(h->ev_start[fam][used], h->s));
  return MG_OK;
}

mg_status prof_end(mg_hierarchy* h, int fam, long long cells) {
  h->stats.launches[fam] += 1;
  h->stats.cells[fam] += cells;
  if (!(h->prof_mask & (1u << fam))) return MG_OK;
  size_t& used = h->ev_used[fam];
  CK(cudaEventRecord(h->ev_end[fam][used], h->s));
  used += 1;
  return MG_OK;
}

// Launch a kernel of family `fam` that processes `cells` cells, counted and
// (when profiling is on for the family) bracketed by CUDA events.
#define KL(fam, cells, expr)              \
  do {                                    \
    ST(prof_begin(h, (fam)));             \
    CK(expr);                             \
    ST(prof_end(h, (fam), (cells)));      \
  } while (0)

long long cells_of(const Grid& G) { return (long long)G.n0 * G.n1 * G.n2; }
long long cells_of(Int3 c) { return (long long)c.x * c.y * c.z; }
long long shell_of(const Grid& G) {
  return (long long)G.X * G.Y * (G.n2 + 2 * G.g) - cells_of(G);
}

bool validate(const mg_config* cfg, char* msg, size_t len, Plan* plan) {
  if (!cfg) {
    if (msg && len) snprintf(msg, len, "config is NULL");
    return false;
  }
  if (cfg->order != 2 && cfg->order != 4 && cfg->order != 6) {
    if (msg && len) snprintf(msg, len, "order must be 2, 4 or 6 (got %d)", cfg->order);
    return false;
  }
  if (cfg->n_levels < 1 || cfg->n_levels > MG_MAX_LEVELS) {
    if (msg && len) snprintf(msg, len, "n_levels must be in [1, %d]", MG_MAX_LEVELS);
    return false;
  }
  for (int a = 0; a < 3; ++a)
    if (cfg->base_n[a] < 2 || cfg->base_n[a] < cfg->order / 2 || cfg->base_n[a] > 4096) {
      if (msg && len) snprintf(msg, len, "base_n[%d] = %d out of range", a, cfg->base_n[a]);
      return false;
    }
  if (!(cfg->box > 0.0) || !std::isfinite(cfg->box)) {
    if (msg && len) snprintf(msg, len, "box must be positive");
    return false;
  }
  if (cfg->precision != MG_FP64 && cfg->precision != MG_MIXED) {
    if (msg && len) snprintf(msg, len, "unknown precision %d", cfg->precision);
    return false;
  }
  if (cfg->precision == MG_MIXED) {
    if (msg && len) snprintf(msg, len, "MG_MIXED is not available in this build");
    return false;
  }
  if (cfg->nu1 < 0 || cfg->nu2 < 0 || cfg->nu1 + cfg->nu2 < 1 || cfg->nu1 > 16 || cfg->nu2 > 16) {
    if (msg && len) snprintf(msg, len, "nu1, nu2 must be in [0, 16] with nu1 + nu2 >= 1");
    return false;
  }
  if (cfg->max_cycles < 1 || cfg->max_cycles > 1000) {
    if (msg && len) snprintf(msg, len, "max_cycles must be in [1, 1000]");
    return false;
  }
  if (!(cfg->tol >= 0.0) || !std::isfinite(cfg->tol)) {
    if (msg && len) snprintf(msg, len, "tol must be finite and >= 0");
    return false;
  }
  if ((cfg->dev_alloc == nullptr) != (cfg->dev_free == nullptr)) {
    if (msg && len) snprintf(msg, len, "dev_alloc and dev_free must be both set or both NULL");
    return false;
  }
  Plan p;
  if (!build_levels(cfg, p.geo, &p.base, msg, len)) return false;
  // bytes
  const int g = cfg->order / 2;
  size_t bytes = 0;
  long long max_leaf = 0;
  int slots = 0;
  for (size_t l = 0; l < p.geo.size(); ++l) {
    const LevelGeom& lg = p.geo[l];
    const Grid G = make_grid(lg.n[0], lg.n[1], lg.n[2], g);
    const size_t e = (size_t)grid_elems(G) * sizeof(double);
    const bool leaf = (int)l >= p.base;
    bytes += 3 * align_up(e);  // u[0], u[1], ffas
    if (leaf) {
      bytes += align_up(e);  // f
      const long long dense = (long long)lg.n[0] * lg.n[1] * lg.n[2];
      if (dense > max_leaf) max_leaf = dense;
      slots += norm_blocks(G);
    }
    if (l > 0) bytes += align_up((size_t)(lg.n[0] / 2) * (lg.n[1] / 2) * (lg.n[2] / 2) * sizeof(double));
    if (lg.nest) {
      FaceSet fs;
      make_faceset(G, g, &fs);
      bytes += align_up((size_t)fs.base[6] * sizeof(double));
      bytes += align_up((size_t)fs.ebase[6] * sizeof(double));
    }
    if (l == 0) bytes += align_up((size_t)lg.n[0] * lg.n[1] * lg.n[2] * sizeof(double));
  }
  bytes += align_up((size_t)slots * 2 * sizeof(double));
  bytes += align_up(4 * sizeof(double));
  bytes += align_up((size_t)3 * max_leaf * sizeof(double));
  p.bytes = bytes;
  if (plan) *plan = p;
  return true;
}

// ---- level operations -------------------------------------------------------

mg_status tangential(mg_hierarchy* h, int l) {
  DevLevel& L = h->L[l];
  DevLevel& P = h->L[l - 1];
  KL(MG_K_GHOST, L.fs.base[6], launch_cf_tangential<double>(h->cfg.order, L.G, P.G, P.u[P.cur], L.off, L.fs, h->w,
                                  1.0 / P.geo.h, L.inter, L.fc_unc, h->s));
  return MG_OK;
}

mg_status ghost_fill(mg_hierarchy* h, int l, bool edges) {
  DevLevel& L = h->L[l];
  if (L.periodic) {
    if (L.ghosts_stale)
      KL(MG_K_GHOST, shell_of(L.G), launch_ghost_periodic<double>(L.G, L.u[L.cur], h->s));
    L.ghosts_stale = false;
    return MG_OK;
  }
  DevLevel& P = h->L[l - 1];
  KL(MG_K_GHOST, 4 * L.fs.ebase[6] * L.G.g, launch_cf_flux<double>(h->cfg.order, L.G, L.u[L.cur], L.fs, h->w, L.inter, L.fc_unc,
                            L.geo.h, 1.0 / L.geo.h, 1.0 / P.geo.h, 1, h->s));
  if (edges)
    KL(MG_K_GHOST, shell_of(L.G), launch_cf_edges<double>(h->cfg.order, L.G, L.u[L.cur], P.G, P.u[P.cur], L.off, h->w, h->s));
  return MG_OK;
}

mg_status half_sweep(mg_hierarchy* h, int l, int colour) {
  DevLevel& L = h->L[l];
  ST(ghost_fill(h, l, false));
  const double a_f = L.geo.h * L.geo.h / centre_weight(h->cfg.order);
  KL(MG_K_SMOOTH, (cells_of(L.G) + 1) / 2, launch_smooth_half<double>(h->cfg.order, L.G, L.u[L.cur], L.u[1 - L.cur], L.ffas, a_f,
                                colour, L.periodic ? 1 : 0, h->s));
  L.cur ^= 1;
  return MG_OK;
}

mg_status smooth(mg_hierarchy* h, int l, int sweeps) {
  for (int s = 0; s < sweeps; ++s) {
    ST(half_sweep(h, l, 0));
    ST(half_sweep(h, l, 1));
  }
  return MG_OK;
}

mg_status vcycle(mg_hierarchy* h, int l) {
  DevLevel& L = h->L[l];
  const int order = h->cfg.order;
  if (l == 0) {
    KL(MG_K_COARSEST, cells_of(L.G), launch_coarsest(L.G, L.ffas, L.u[L.cur], L.kern, h->s));
    return MG_OK;
  }
  DevLevel& P = h->L[l - 1];
  ST(smooth(h, l, h->cfg.nu1));
  ST(ghost_fill(h, l, false));
  KL(MG_K_RESTRICT, cells_of(L.G), launch_residual_restrict<double>(order, L.G, L.u[L.cur], L.ffas, 1.0 / (L.geo.h * L.geo.h),
                                      P.G, P.u[P.cur], P.ffas, L.ubar, L.off, L.cn,
                                      P.periodic ? 1 : 0, h->s));
  KL(MG_K_FAS, cells_of(L.cn), launch_fas_source<double>(order, P.G, P.u[P.cur], P.ffas, 1.0 / (P.geo.h * P.geo.h), L.off,
                               L.cn, h->s));
  ST(vcycle(h, l - 1));
  if (!L.periodic) ST(tangential(h, l));
  KL(MG_K_PROLONG, cells_of(L.G), launch_prolong<double>(L.G, L.u[L.cur], P.G, P.u[P.cur], L.ubar, L.off, L.cn,
                                 L.periodic ? 1 : 0, h->s));
  ST(smooth(h, l, h->cfg.nu2));
  return MG_OK;
}

int finest(const mg_hierarchy* h) { return (int)h->L.size() - 1; }

mg_status sync_covered(mg_hierarchy* h) {
  for (int l = finest(h); l > h->base; --l) {
    DevLevel& L = h->L[l];
    DevLevel& P = h->L[l - 1];
    KL(MG_K_RESTRICT, cells_of(L.G), launch_restrict_u<double>(L.G, L.u[L.cur], P.G, P.u[P.cur], L.off, L.cn, h->s));
  }
  return MG_OK;
}

// Leaf residual norm after syncing covered cells; reads 4 doubles back.
mg_status leaf_norms(mg_hierarchy* h, double* rr, double* ff, double* fsum) {
  ST(sync_covered(h));
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    ST(ghost_fill(h, l, false));
    KL(MG_K_NORM, cells_of(L.G), launch_norm_partial(h->cfg.order, L.G, L.u[L.cur], L.f, 1.0 / (L.geo.h * L.geo.h),
                           L.geo.h * L.geo.h * L.geo.h, L.child_lo, L.child_hi,
                           h->partial + 2 * L.partial_off, L.nblocks, h->s));
  }
  KL(MG_K_NORM, h->partial_slots, launch_reduce_partials(h->partial, h->partial_slots, 2, h->red, h->s));
  CK(cudaMemcpyAsync(h->host_red, h->red, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  *rr = h->host_red[0];
  *ff = h->host_red[1];
  if (fsum) *fsum = h->host_red[2];
  return MG_OK;
}

// f on leaf levels holds the source; removes the composite mean, runs V-cycles.
mg_status solve_prepared(mg_hierarchy* h, mg_info* info) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    KL(MG_K_NORM, cells_of(L.G), launch_sum_partial(L.G, L.f, L.geo.h * L.geo.h * L.geo.h, L.child_lo, L.child_hi,
                          h->partial + 2 * L.partial_off, L.nblocks, h->s));
  }
  KL(MG_K_NORM, h->partial_slots, launch_reduce_partials(h->partial, h->partial_slots, 2, h->red + 2, h->s));
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    KL(MG_K_COPY, cells_of(L.G), launch_shift_copy(L.G, L.f, L.ffas, h->red + 2, 1.0 / h->volume, h->s));
  }
  for (size_t l = 0; l < h->L.size(); ++l) {
    DevLevel& L = h->L[l];
    const long long e = grid_elems(L.G);
    KL(MG_K_COPY, e, launch_fill(L.u[0], e, 0.0, h->s));
    KL(MG_K_COPY, e, launch_fill(L.u[1], e, 0.0, h->s));
    L.cur = 0;
    L.ghosts_stale = false;
  }
  for (int l = h->base + 1; l <= finest(h); ++l) ST(tangential(h, l));
  mg_info local;
  std::memset(&local, 0, sizeof(local));
  double rel = INFINITY;
  const bool fixed = !(h->cfg.tol > 0.0);
  for (int c = 0; c < h->cfg.max_cycles; ++c) {
    ST(vcycle(h, finest(h)));
    double rr, ff, fs;
    ST(leaf_norms(h, &rr, &ff, &fs));
    if (c == 0) local.source_mean = fs / h->volume;
    rel = ff > 0.0 ? std::sqrt(rr) / std::sqrt(ff) : std::sqrt(rr);
    if (local.cycles < MG_MAX_HISTORY) local.history[local.cycles] = rel;
    local.cycles++;
    if (!std::isfinite(rel)) break;
    if (!fixed && rel <= h->cfg.tol) break;
  }
  local.rel_residual = rel;
  if (info) *info = local;
  if (!std::isfinite(rel)) return fail(h, MG_ENOCONV, "residual is not finite");
  if (!fixed && rel > h->cfg.tol) return fail(h, MG_ENOCONV, "max_cycles reached above tol");
  return MG_OK;
}

cudaMemcpy3DParms dense_padded_parms(const DevLevel& L, double* padded, double* dense,
                                     bool to_padded) {
  cudaMemcpy3DParms p;
  std::memset(&p, 0, sizeof(p));
  const Grid& G = L.G;
  cudaPitchedPtr pp = make_cudaPitchedPtr(padded, (size_t)G.Zp * sizeof(double),
                                          (size_t)G.Zp * sizeof(double), (size_t)G.Y);
  cudaPitchedPtr dp = make_cudaPitchedPtr(dense, (size_t)G.n2 * sizeof(double),
                                          (size_t)G.n2 * sizeof(double), (size_t)G.n1);
  cudaPos ppos = make_cudaPos((size_t)G.za * sizeof(double), (size_t)G.g, (size_t)G.g);
  if (to_padded) {
    p.srcPtr = dp;
    p.dstPtr = pp;
    p.dstPos = ppos;
  } else {
    p.srcPtr = pp;
    p.srcPos = ppos;
    p.dstPtr = dp;
  }
  p.extent = make_cudaExtent((size_t)G.n2 * sizeof(double), (size_t)G.n1, (size_t)G.n0);
  p.kind = cudaMemcpyDefault;
  return p;
}

mg_status load_leaf(mg_hierarchy* h, int l, const double* src, double* padded, bool host) {
  DevLevel& L = h->L[l];
  if (host) {
    cudaMemcpy3DParms p = dense_padded_parms(L, padded, const_cast<double*>(src), true);
    CK(cudaMemcpy3DAsync(&p, h->s));
  } else {
    KL(MG_K_COPY, cells_of(L.G), launch_pack(L.G, src, padded, 0.0, h->s));
  }
  return MG_OK;
}

mg_status store_leaf(mg_hierarchy* h, int l, const double* padded, double* dst, bool host) {
  DevLevel& L = h->L[l];
  if (host) {
    cudaMemcpy3DParms p = dense_padded_parms(L, const_cast<double*>(padded), dst, false);
    CK(cudaMemcpy3DAsync(&p, h->s));
  } else {
    KL(MG_K_COPY, cells_of(L.G), launch_unpack(L.G, padded, dst, h->s));
  }
  return MG_OK;
}

// phi (dense per leaf level) -> u[cur]; covered cells := mean of children.
mg_status load_potential(mg_hierarchy* h, const double* const phi[], bool host) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    ST(load_leaf(h, l, phi[l - h->base], L.u[L.cur], host));
    L.ghosts_stale = true;
  }
  ST(sync_covered(h));
  for (int l = h->base + 1; l <= finest(h); ++l) ST(tangential(h, l));
  return MG_OK;
}

// tau of the potential currently in u[cur] into f of every leaf level.
mg_status tau_into_f(mg_hierarchy* h) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    ST(ghost_fill(h, l, true));
    KL(MG_K_LPT, cells_of(L.G), launch_lpt2_source(h->cfg.order, L.G, L.u[L.cur], 1.0 / (L.geo.h * L.geo.h), L.f, h->s));
  }
  for (int l = finest(h); l > h->base; --l) {
    DevLevel& L = h->L[l];
    DevLevel& P = h->L[l - 1];
    KL(MG_K_RESTRICT, cells_of(L.G), launch_restrict_u<double>(L.G, L.f, P.G, P.f, L.off, L.cn, h->s));
  }
  return MG_OK;
}

// -G phi of the potential in u[cur]; outputs dense, 3 per leaf level.
mg_status gradient_out(mg_hierarchy* h, double* const disp[], bool host) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    const int i = l - h->base;
    ST(ghost_fill(h, l, false));
    double* dx = disp[3 * i];
    double* dy = disp[3 * i + 1];
    double* dz = disp[3 * i + 2];
    const long long n = (long long)L.G.n0 * L.G.n1 * L.G.n2;
    if (host) {
      if (!dx && !dy && !dz) continue;
      KL(MG_K_LPT, n, launch_gradient(h->cfg.order, L.G, L.u[L.cur], 1.0 / L.geo.h, h->scratch,
                         h->scratch + n, h->scratch + 2 * n, h->s));
      for (int a = 0; a < 3; ++a)
        if (disp[3 * i + a])
          CK(cudaMemcpyAsync(disp[3 * i + a], h->scratch + a * n, n * sizeof(double),
                             cudaMemcpyDeviceToHost, h->s));
    } else {
      if (!dx || !dy || !dz) return fail(h, MG_EINVAL, "displacement output pointer is NULL");
      KL(MG_K_LPT, n, launch_gradient(h->cfg.order, L.G, L.u[L.cur], 1.0 / L.geo.h, dx, dy, dz, h->s));
    }
  }
  return MG_OK;
}

bool check_ptrs(mg_hierarchy* h, const void* const* p, int count) {
  if (!p) return false;
  for (int i = 0; i < count; ++i)
    if (!p[i]) return false;
  (void)h;
  return true;
}

int n_leaf(const mg_hierarchy* h) { return (int)h->L.size() - h->base; }

}  // namespace

// ---- C ABI -------------------------------------------------------------------

extern "C" {

void mg_config_default(mg_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n_levels = 1;
  cfg->base_n[0] = cfg->base_n[1] = cfg->base_n[2] = 64;
  cfg->box = 1.0;
  cfg->order = 2;
  cfg->precision = MG_FP64;
  cfg->nu1 = 2;
  cfg->nu2 = 2;
  cfg->max_cycles = 50;
  cfg->tol = 1e-10;
}

mg_status mg_config_validate(const mg_config* cfg, char* msg, size_t len) {
  if (msg && len) msg[0] = '\0';
  return validate(cfg, msg, len, nullptr) ? MG_OK : MG_EINVAL;
}

size_t mg_workspace_bytes(const mg_config* cfg) {
  Plan p;
  if (!validate(cfg, nullptr, 0, &p)) return 0;
  return p.bytes;
}

int mg_total_levels(const mg_config* cfg) {
  Plan p;
  if (!validate(cfg, nullptr, 0, &p)) return 0;
  return (int)p.geo.size();
}

const char* mg_version(void) { return "mgic-gb300 0.1 (sm_103a)"; }

mg_status mg_set_profiling(mg_hierarchy* h, unsigned mask) {
  if (!h) return MG_EINVAL;
  h->prof_mask = mask & ((1u << MG_K_FAMILIES) - 1u);
  return MG_OK;
}

mg_status mg_get_stats(mg_hierarchy* h, mg_stats* out, int reset) {
  if (!h || !out) return MG_EINVAL;
  CK(cudaStreamSynchronize(h->s));
  for (int f = 0; f < MG_K_FAMILIES; ++f) {
    for (size_t i = 0; i < h->ev_used[f]; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->ev_start[f][i], h->ev_end[f][i]));
      h->stats.event_ms[f] += ms;
    }
    h->stats.timed[f] += (long long)h->ev_used[f];
    h->ev_used[f] = 0;
  }
  *out = h->stats;
  if (reset) std::memset(&h->stats, 0, sizeof(h->stats));
  return MG_OK;
}

const char* mg_last_error(const mg_hierarchy* h) { return h ? h->err.c_str() : ""; }

mg_status mg_hierarchy_create(const mg_config* cfg, void* cuda_stream, mg_hierarchy** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  Plan plan;
  char msg[256];
  if (!validate(cfg, msg, sizeof(msg), &plan)) return MG_EINVAL;
  mg_hierarchy* h = new mg_hierarchy();
  std::memset(&h->stats, 0, sizeof(h->stats));
  h->cfg = *cfg;
  h->s = (cudaStream_t)cuda_stream;
  h->base = plan.base;
  const int order = cfg->order;
  const int g = order / 2;
  compute_cf_weights(order, &h->w);
  // allocate
  if (cfg->dev_alloc) {
    h->arena = cfg->dev_alloc(plan.bytes, cfg->alloc_ctx);
    if (!h->arena) {
      delete h;
      return MG_ENOMEM;
    }
  } else {
    cudaError_t e = cudaMalloc(&h->arena, plan.bytes);
    if (e != cudaSuccess) {
      delete h;
      return e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA;
    }
  }
  h->arena_bytes = plan.bytes;
  char* cursor = (char*)h->arena;
  auto take = [&](size_t bytes) {
    char* p = cursor;
    cursor += align_up(bytes);
    return (double*)p;
  };
  const size_t nl = plan.geo.size();
  h->L.resize(nl);
  int slots = 0;
  long long max_leaf = 0;
  for (size_t l = 0; l < nl; ++l) {
    DevLevel& L = h->L[l];
    L.geo = plan.geo[l];
    L.G = make_grid(L.geo.n[0], L.geo.n[1], L.geo.n[2], g);
    L.periodic = !L.geo.nest;
    L.leaf = (int)l >= h->base;
    L.has_child = l + 1 < nl;
    L.off = Int3{L.geo.off[0], L.geo.off[1], L.geo.off[2]};
    L.cn = Int3{L.geo.n[0] / 2, L.geo.n[1] / 2, L.geo.n[2] / 2};
    const size_t e = (size_t)grid_elems(L.G) * sizeof(double);
    L.u[0] = take(e);
    L.u[1] = take(e);
    L.ffas = take(e);
    if (L.leaf) {
      L.f = take(e);
      const long long dense = (long long)L.geo.n[0] * L.geo.n[1] * L.geo.n[2];
      if (dense > max_leaf) max_leaf = dense;
      L.nblocks = norm_blocks(L.G);
      L.partial_off = slots;
      slots += L.nblocks;
    }
    if (l > 0) L.ubar = take((size_t)L.cn.x * L.cn.y * L.cn.z * sizeof(double));
    if (L.geo.nest) {
      make_faceset(L.G, g, &L.fs);
      L.inter = take((size_t)L.fs.base[6] * sizeof(double));
      L.fc_unc = take((size_t)L.fs.ebase[6] * sizeof(double));
    }
    if (l == 0) L.kern = take((size_t)L.geo.n[0] * L.geo.n[1] * L.geo.n[2] * sizeof(double));
  }
  for (size_t l = 0; l + 1 < nl; ++l) {
    DevLevel& L = h->L[l];
    const DevLevel& C = h->L[l + 1];
    if (L.leaf) {
      L.child_lo = C.off;
      L.child_hi = Int3{C.off.x + C.cn.x, C.off.y + C.cn.y, C.off.z + C.cn.z};
    }
  }
  h->partial_slots = slots;
  h->partial = take((size_t)slots * 2 * sizeof(double));
  h->red = take(4 * sizeof(double));
  h->scratch_elems = max_leaf;
  h->scratch = take((size_t)3 * max_leaf * sizeof(double));
  const LevelGeom& b = plan.geo[plan.base];
  h->volume = b.h * b.h * b.h * (double)b.n[0] * b.n[1] * b.n[2];
  cudaError_t e = cudaMallocHost(&h->host_red, 4 * sizeof(double));
  if (e != cudaSuccess) {
    mg_hierarchy_destroy(h);
    return MG_ECUDA;
  }
  std::vector<double> K;
  const LevelGeom& c = plan.geo[0];
  coarsest_kernel(order, c.n[0], c.n[1], c.n[2], c.h, K);
  e = cudaMemcpyAsync(h->L[0].kern, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice,
                      h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  if (e != cudaSuccess) {
    mg_hierarchy_destroy(h);
    return MG_ECUDA;
  }
  *out = h;
  return MG_OK;
}

mg_status mg_hierarchy_destroy(mg_hierarchy* h) {
  if (!h) return MG_OK;
  if (h->s) cudaStreamSynchronize(h->s);
  else cudaDeviceSynchronize();
  if (h->arena) {
    if (h->cfg.dev_free) h->cfg.dev_free(h->arena, h->cfg.alloc_ctx);
    else cudaFree(h->arena);
  }
  if (h->host_red) cudaFreeHost(h->host_red);
  for (int f = 0; f < MG_K_FAMILIES; ++f) {
    for (cudaEvent_t e : h->ev_start[f]) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_end[f]) cudaEventDestroy(e);
  }
  delete h;
  return MG_OK;
}

mg_status mg_solve_1lpt(mg_hierarchy* h, const double* const delta[], double* const phi[],
                        mg_info* info) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs(h, (const void* const*)delta, nleaf) || !check_ptrs(h, (const void* const*)phi, nleaf))
    return fail(h, MG_EINVAL, "delta/phi must hold one non-NULL pointer per level");
  for (int l = h->base; l <= finest(h); ++l) ST(load_leaf(h, l, delta[l - h->base], h->L[l].f, false));
  const mg_status st = solve_prepared(h, info);
  if (st != MG_OK && st != MG_ENOCONV) return st;
  for (int l = h->base; l <= finest(h); ++l)
    ST(store_leaf(h, l, h->L[l].u[h->L[l].cur], phi[l - h->base], false));
  CK(cudaStreamSynchronize(h->s));
  return st;
}

mg_status mg_lpt2_source(mg_hierarchy* h, const double* const phi1[], double* const tau[]) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs(h, (const void* const*)phi1, nleaf) || !check_ptrs(h, (const void* const*)tau, nleaf))
    return fail(h, MG_EINVAL, "phi1/tau must hold one non-NULL pointer per level");
  ST(load_potential(h, phi1, false));
  ST(tau_into_f(h));
  for (int l = h->base; l <= finest(h); ++l) ST(store_leaf(h, l, h->L[l].f, tau[l - h->base], false));
  CK(cudaStreamSynchronize(h->s));
  return MG_OK;
}

mg_status mg_solve_2lpt(mg_hierarchy* h, const double* const phi1[], double* const phi2[],
                        mg_info* info) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs(h, (const void* const*)phi1, nleaf) || !check_ptrs(h, (const void* const*)phi2, nleaf))
    return fail(h, MG_EINVAL, "phi1/phi2 must hold one non-NULL pointer per level");
  ST(load_potential(h, phi1, false));
  ST(tau_into_f(h));
  const mg_status st = solve_prepared(h, info);
  if (st != MG_OK && st != MG_ENOCONV) return st;
  for (int l = h->base; l <= finest(h); ++l)
    ST(store_leaf(h, l, h->L[l].u[h->L[l].cur], phi2[l - h->base], false));
  CK(cudaStreamSynchronize(h->s));
  return st;
}

mg_status mg_displacements(mg_hierarchy* h, const double* const phi[], double* const disp[]) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs(h, (const void* const*)phi, nleaf) || !check_ptrs(h, (const void* const*)disp, 3 * nleaf))
    return fail(h, MG_EINVAL, "phi/disp must hold 1 and 3 non-NULL pointers per level");
  ST(load_potential(h, phi, false));
  ST(gradient_out(h, disp, false));
  CK(cudaStreamSynchronize(h->s));
  return MG_OK;
}

mg_status mg_lpt_pipeline(mg_hierarchy* h, int host_buffers, const double* const delta[],
                          double* const phi1[], double* const phi2[], double* const disp1[],
                          double* const disp2[], mg_info* info1, mg_info* info2) {
  if (!h) return MG_EINVAL;
  const bool host = host_buffers != 0;
  const int nleaf = n_leaf(h);
  if (!check_ptrs(h, (const void* const*)delta, nleaf))
    return fail(h, MG_EINVAL, "delta must hold one non-NULL pointer per level");
  if (!host) {
    if (!check_ptrs(h, (const void* const*)disp1, 3 * nleaf) ||
        !check_ptrs(h, (const void* const*)disp2, 3 * nleaf))
      return fail(h, MG_EINVAL, "device displacement outputs must all be set");
  }
  for (int l = h->base; l <= finest(h); ++l) ST(load_leaf(h, l, delta[l - h->base], h->L[l].f, host));
  mg_status st1 = solve_prepared(h, info1);
  if (st1 != MG_OK && st1 != MG_ENOCONV) return st1;
  if (phi1)
    for (int l = h->base; l <= finest(h); ++l)
      if (phi1[l - h->base]) ST(store_leaf(h, l, h->L[l].u[h->L[l].cur], phi1[l - h->base], host));
  if (disp1) ST(gradient_out(h, disp1, host));
  ST(tau_into_f(h));
  mg_status st2 = solve_prepared(h, info2);
  if (st2 != MG_OK && st2 != MG_ENOCONV) return st2;
  if (phi2)
    for (int l = h->base; l <= finest(h); ++l)
      if (phi2[l - h->base]) ST(store_leaf(h, l, h->L[l].u[h->L[l].cur], phi2[l - h->base], host));
  if (disp2) ST(gradient_out(h, disp2, host));
  CK(cudaStreamSynchronize(h->s));
  return st1 != MG_OK ? st1 : st2;
}

}  // extern "C"
