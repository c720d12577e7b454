// Hierarchy object, FAS V-cycle driver and the C ABI of include/mg.h.
//
// The V-cycle follows Hahn & Abel 2011, Sec. 3.2 (enumerated algorithm) on the
// composite grid of Sec. 3.3: levels below the base are full periodic
// coarsenings, the base is periodic, nests take their boundary values from
// the parent through coarse-fine interpolation with flux matching.  Every step
// is a kernel launch on the hierarchy's stream; the host only sequences them
// and reads back one convergence record per cycle.
//
// Precision.  MG_FP64 runs the V-cycle on float64 buffers.  MG_MIXED keeps a
// float64 solution on the leaf levels only; each outer iteration computes the
// float64 composite residual r = f - L u (which also gives the convergence
// norm), solves L e = r from e = 0 with float32 V-cycles on float32 buffers of
// every level (the same kernels instantiated for float; coarse-fine ghosts,
// flux matching and restriction are linear, so the correction equation has
// the same composite operator), and adds e to u in float64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cfloat>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "mg.h"
#include "mg_internal.h"
#include "mg_persist.h"
#include "mg_setup.h"

using namespace mgk;

namespace {

// Working buffers of one level in one precision.
template <typename T>
struct Bufs {
  T* u[2] = {nullptr, nullptr};  // smoother double buffer; u[cur] is current
  int cur = 0;
  T* ffas = nullptr;             // working source
  T* ubar = nullptr;             // restricted copy of this level's u (levels with a parent)
  T* inter = nullptr;            // nests: tangential intermediate values
  T* fc_unc = nullptr;           // nests: uncovered part of the parent face flux
  // Periodic levels: every kernel that writes u also writes its ghost images,
  // so ghosts are refilled only after u is loaded from outside.
  bool ghosts_stale = true;
  // TMA-staged smoother: tensor maps of u[0], u[1] and ffas
  bool tma = false;
  CUtensorMap tm[2];
  CUtensorMap tm_f;
};

struct DevLevel {
  LevelGeom geo;
  Grid G;
  bool periodic = true;
  bool leaf = false;
  Int3 off{0, 0, 0};  // origin in parent cells
  Int3 cn{0, 0, 0};   // covered extent in the parent
  Int3 child_lo{0, 0, 0}, child_hi{0, 0, 0};  // region covered by the child, own cells
  Bufs<double> d;     // float64 state (MG_FP64: every level; MG_MIXED: leaf levels, u[0] only)
  Bufs<float> s;      // float32 correction state (MG_MIXED only)
  double* f = nullptr;     // leaf levels: float64 source
  double* kern = nullptr;  // coarsest level: periodic pseudo-inverse kernel
  FaceSet fs;
  int nblocks = 0;
  int partial_off = 0;
  long long stage_off = 0;  // leaf levels: offset of the level's 4 dense arrays in stage
};

template <typename T>
Bufs<T>& bufs(DevLevel& L);
template <>
Bufs<double>& bufs<double>(DevLevel& L) {
  return L.d;
}
template <>
Bufs<float>& bufs<float>(DevLevel& L) {
  return L.s;
}

constexpr size_t kAlign = 256;
// doubles of the reduction record: norm sums, source sum, wait flag, per-level norm sums
constexpr int kRedDoubles = 8 + 2 * MG_MAX_LEVELS;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

double centre_weight(int order) {
  double l[7];
  laplacian_1d(order, l);
  return 3.0 * l[order / 2];
}

// Carves the arena; with base == nullptr it only counts bytes.
struct Carver {
  char* base = nullptr;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += align_up(count * sizeof(T));
    return p;
  }
};

// A CUDA-event pair recorded around one timed launch inside a captured graph.
struct ProfEv {
  int fam;
  cudaEvent_t a, b;
  long long cells;
};

// One captured and instantiated cycle body with the launch counts it adds per
// replay and the event pairs it records.
struct Graph {
  cudaGraphExec_t exec = nullptr;
  unsigned mask = 0;
  long long min_cells = 0;
  mg_stats delta;
  std::vector<ProfEv> evs;
};

}  // namespace

// Kernels of the device-side iteration loop live in a named namespace (kernels in
// this file's anonymous namespace would clash with those of mgk's).
namespace mgloop {

// Convergence record of a solve whose iteration loop runs on the device
// (MG_FLAG_DEVICE_LOOP), written by k_loop_step after every iteration.
struct LoopState {
  int c;            // iterations run
  int done;
  int timeout;      // a smoother block's bounded wait ran out
  int at_floor;     // residual at the rounding level of the source
  int inner_now;    // MG_MIXED: float32 V-cycles of the next outer iteration
  int inner_total;  // MG_MIXED: float32 V-cycles run
  double rel;       // relative leaf residual after the last iteration
  double source_mean;
  double history[MG_MAX_HISTORY];
  unsigned char inner_hist[MG_MAX_HISTORY];  // MG_MIXED: inner cycles per iteration
  double level_rel[MG_MAX_LEVELS];           // per leaf level, after the last iteration
};

// The relative residual of one leaf level from its volume-weighted sums of r^2 and f^2
// (the residual norm itself when the level's source is zero).
__host__ __device__ inline double level_relative(double rr, double ff) {
  return ff > 0.0 ? sqrt(rr) / sqrt(ff) : sqrt(rr);
}

__host__ __device__ inline int inner_plan(int cap, double tol, double rel_before, double rel_after,
                                          int used) {
  if (!(tol > 0.0) || !(rel_after > 0.0) || !(rel_before > rel_after) || used < 1) return cap;
  const double c = log(5.0);
  const double k = (log(rel_before / rel_after) + c) / used;
  const double need = (log(rel_after / (0.25 * tol)) + c) / k;
  if (!(need == need) || need > 1e9 || need < -1e9) return cap;
  const int n = (int)ceil(need);
  return n < 1 ? 1 : (n > cap ? cap : n);
}

struct LoopParams {
  double tol;
  double volume;
  int max_cycles;
  int mixed;
  int cap;
  int n_leaf;  // leaf levels (base and nests): red[8 + 2 l], red[9 + 2 l] hold level l's sums
};

__global__ void k_loop_init(LoopState* st, int mixed, int cap) {
  st->c = 0;
  st->done = 0;
  st->timeout = 0;
  st->at_floor = 0;
  st->inner_now = cap;
  st->inner_total = 0;
  // MG_MIXED starts from u = 0, whose residual is the source itself
  st->rel = mixed ? 1.0 : INFINITY;
  st->source_mean = 0.0;
}

// After iteration st->c: the same record and stopping rule as solve_step_read.
__global__ void k_loop_step(LoopState* st, const double* red, LoopParams p,
                            cudaGraphConditionalHandle while_h, cudaGraphConditionalHandle switch_h) {
  const double rr = red[0], ff = red[1], fs = red[2];
  const unsigned flag = *reinterpret_cast<const unsigned*>(red + 4);
  const int c = st->c;
  if (c == 0) st->source_mean = fs / p.volume;
  const double before = st->rel;
  const double rel = ff > 0.0 ? sqrt(rr) / sqrt(ff) : sqrt(rr);
  st->rel = rel;
  if (p.mixed) {
    st->inner_total += st->inner_now;
    if (c < MG_MAX_HISTORY) st->inner_hist[c] = (unsigned char)st->inner_now;
    st->inner_now = inner_plan(p.cap, p.tol, before, rel, st->inner_now);
  }
  if (c < MG_MAX_HISTORY) st->history[c] = rel;
  for (int l = 0; l < p.n_leaf; ++l) st->level_rel[l] = level_relative(red[8 + 2 * l], red[9 + 2 * l]);
  st->c = c + 1;
  const bool fixed = !(p.tol > 0.0);
  const double mean = st->source_mean;
  const double floor_ = 64.0 * DBL_EPSILON * sqrt(ff + p.volume * mean * mean);
  const bool at_floor = !fixed && sqrt(rr) <= floor_;
  const bool finite = rel == rel && rel < INFINITY;
  const bool done = !finite || (!fixed && rel <= p.tol) || at_floor || c + 1 >= p.max_cycles ||
                    flag != 0;
  st->at_floor = at_floor ? 1 : 0;
  st->timeout = flag != 0 ? 1 : 0;
  st->done = done ? 1 : 0;
  cudaGraphSetConditional(while_h, done ? 0u : 1u);
  if (p.mixed) cudaGraphSetConditional(switch_h, (unsigned)(st->inner_now - 1));
}

}  // namespace mgloop

using mgloop::LoopState;

namespace {

struct LoopGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  mg_stats body[17];  // launches of one iteration: [0] FP64 V-cycle + norm;
                      // MG_MIXED: [n] zero correction + n float32 V-cycles
  mg_stats tail;      // MG_MIXED: update, ghosts and norm after the inner cycles
};

}  // namespace

struct mg_hierarchy {
  mg_config cfg;
  std::vector<DevLevel> L;
  int base = 0;
  bool mixed = false;
  cudaStream_t user_s = nullptr;  // the caller's stream
  cudaStream_t s = nullptr;       // the hierarchy's own non-blocking work stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // MG_FP64: V-cycle + norm; MG_MIXED: outer iteration + norm.  [0] launches
  // plainly; [1] also records the profiling events (first cycle of each solve).
  // [inner cycles of the body (MG_MIXED; 0 for MG_FP64)][timed]
  Graph g_cycle[17][2];
  int inner_now = 0;  // MG_MIXED: float32 V-cycles of the next outer iteration
  Graph* capturing = nullptr;     // graph being captured
  Graph* replayed = nullptr;      // graph whose event pairs await reading
  // when set, the float32 level operations are appended here (a work list for the
  // persistent batch kernel) instead of being launched; the host-side state (buffer
  // parities, stale flags) advances exactly as for launches
  std::vector<mgk::POp>* rec = nullptr;
  CfWeights w;
  std::string err;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  double* partial = nullptr;
  int partial_slots = 0;
  // [0..1] norm sums, [2..3] source sum, [4] wait flag, [8 + 2 l, 9 + 2 l] the norm
  // sums of leaf level l (kRedDoubles in all)
  double* red = nullptr;
  double* host_red = nullptr;  // pinned copy of red
  unsigned* wait_err = nullptr;  // device flag: a bounded wait in a kernel ran out
  double* scratch = nullptr;   // 3 dense arrays of the largest leaf level
  long long scratch_elems = 0;
  double* tau_work = nullptr;  // 3 padded float64 arrays of the largest leaf level
  // host-buffer pipelines: the first solve's phi and displacements are staged here
  // (phi, x, y, z per leaf level, dense) and copied to the host on cs while the
  // second solve runs
  double* stage = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_staged = nullptr, ev_copied = nullptr;
  bool copies_pending = false;
  // hybrid Poisson correction of the finest level (MG_FLAG_HYBRID), made on first use
  HybridFFT* hybrid = nullptr;
  double* hybrid_f = nullptr;  // dense source of the finest level
  double volume = 0.0;
  // device-side iteration loop (MG_FLAG_DEVICE_LOOP), built on first use
  LoopGraph loop;
  LoopState* loop_dev = nullptr;
  LoopState* loop_host = nullptr;  // pinned copy written at the end of the loop graph
  LoopState* loop_host1 = nullptr;  // pinned: the first solve's record in a pipeline
  // launch counters and optional CUDA-event timing per kernel family
  mg_stats stats;
  unsigned prof_mask = 0;    // families the caller asked to time
  unsigned active_mask = 0;  // families timed by the launches being issued now
  long long prof_min_cells = 0;  // only launches of at least this many cells are timed
  std::vector<cudaEvent_t> ev_start[MG_K_FAMILIES], ev_end[MG_K_FAMILIES];
  std::vector<long long> ev_cells[MG_K_FAMILIES];
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

bool prof_on(const mg_hierarchy* h, int fam, long long cells) {
  return (h->active_mask & (1u << fam)) && cells >= h->prof_min_cells;
}

mg_status prof_begin(mg_hierarchy* h, int fam, long long cells) {
  if (!prof_on(h, fam, cells)) return MG_OK;
  if (h->capturing) {
    ProfEv ev{fam, nullptr, nullptr, cells};
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    h->capturing->evs.push_back(ev);
    CK(cudaEventRecordWithFlags(ev.a, h->s, cudaEventRecordExternal));
    return MG_OK;
  }
  size_t& used = h->ev_used[fam];
  if (used == h->ev_start[fam].size()) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    h->ev_start[fam].push_back(a);
    h->ev_end[fam].push_back(b);
    h->ev_cells[fam].push_back(0);
  }
  h->ev_cells[fam][used] = cells;
  CK(cudaEventRecord(h->ev_start[fam][used], h->s));
  return MG_OK;
}

mg_status prof_end(mg_hierarchy* h, int fam, long long cells) {
  h->stats.launches[fam] += 1;
  h->stats.cells[fam] += cells;
  if (!prof_on(h, fam, cells)) return MG_OK;
  if (h->capturing) {
    CK(cudaEventRecordWithFlags(h->capturing->evs.back().b, h->s, cudaEventRecordExternal));
    return MG_OK;
  }
  size_t& used = h->ev_used[fam];
  CK(cudaEventRecord(h->ev_end[fam][used], h->s));
  used += 1;
  return MG_OK;
}

// Launch a kernel of family `fam` that processes `cells` cells, counted and
// (when profiling is on for the family) bracketed by CUDA events.
#define KL(fam, cells, expr)              \
  do {                                    \
    ST(prof_begin(h, (fam), (cells)));    \
    CK(expr);                             \
    ST(prof_end(h, (fam), (cells)));      \
  } while (0)

long long cells_of(const Grid& G) { return (long long)G.n0 * G.n1 * G.n2; }

// ---- work-list recording (persistent batch kernel) -----------------------------

template <typename T>
bool recording(const mg_hierarchy* h) {
  return std::is_same<T, float>::value && h->rec != nullptr;
}

// Appends an operation of nblk blocks; 3D operations give their grid's x and y extents.
void rec_push(mg_hierarchy* h, POp op, long long nblk, int gx = 1, int gy = 1) {
  op.nblk = (int)nblk;
  op.gx = gx;
  op.gy = gy;
  // about 1024 work items per operation at most: few atomics, enough items to spread
  op.per_tile = (int)(nblk > 1024 ? (nblk + 1023) / 1024 : 1);
  op.ntiles = (int)((nblk + op.per_tile - 1) / op.per_tile);
  op.order = h->cfg.order;
  if (nblk > 0) h->rec->push_back(op);
}

POp pop(int kind) {
  POp o;
  std::memset(&o, 0, sizeof(o));
  o.kind = kind;
  return o;
}

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }
long long cells_of(Int3 c) { return (long long)c.x * c.y * c.z; }
long long shell_of(const Grid& G) {
  return (long long)G.X * G.Y * (G.n2 + 2 * G.g) - cells_of(G);
}

struct Plan {
  std::vector<LevelGeom> geo;
  int base = 0;
  size_t bytes = 0;
};

// Lays out every buffer of the hierarchy (counting only when h == nullptr).
size_t carve(const mg_config* cfg, const Plan& p, mg_hierarchy* h, char* arena) {
  Carver c;
  c.base = arena;
  const int g = cfg->order / 2;
  const bool mixed = cfg->precision == MG_MIXED;
  int slots = 0;
  long long leaf_total = 0;
  long long max_leaf = 0;
  long long max_leaf_padded = 0;
  const size_t nl = p.geo.size();
  for (size_t l = 0; l < nl; ++l) {
    const LevelGeom& lg = p.geo[l];
    const Grid G = make_grid(lg.n[0], lg.n[1], lg.n[2], g);
    const size_t e = (size_t)grid_elems(G);
    const bool leaf = (int)l >= p.base;
    const size_t ncov = (size_t)(lg.n[0] / 2) * (lg.n[1] / 2) * (lg.n[2] / 2);
    FaceSet fs;
    make_faceset(G, g, &fs);
    DevLevel* L = h ? &h->L[l] : nullptr;
    if (!mixed) {
      double* u0 = c.take<double>(e);
      double* u1 = c.take<double>(e);
      double* ff = c.take<double>(e);
      double* ub = l > 0 ? c.take<double>(ncov) : nullptr;
      double* in = lg.nest ? c.take<double>((size_t)fs.base[6]) : nullptr;
      double* fu = lg.nest ? c.take<double>((size_t)fs.ebase[6]) : nullptr;
      if (L) {
        L->d.u[0] = u0;
        L->d.u[1] = u1;
        L->d.ffas = ff;
        L->d.ubar = ub;
        L->d.inter = in;
        L->d.fc_unc = fu;
      }
    } else {
      float* u0 = c.take<float>(e);
      float* u1 = c.take<float>(e);
      float* ff = c.take<float>(e);
      float* ub = l > 0 ? c.take<float>(ncov) : nullptr;
      float* in = lg.nest ? c.take<float>((size_t)fs.base[6]) : nullptr;
      float* fu = lg.nest ? c.take<float>((size_t)fs.ebase[6]) : nullptr;
      if (L) {
        L->s.u[0] = u0;
        L->s.u[1] = u1;
        L->s.ffas = ff;
        L->s.ubar = ub;
        L->s.inter = in;
        L->s.fc_unc = fu;
      }
      if (leaf) {
        double* u0d = c.take<double>(e);
        double* ind = lg.nest ? c.take<double>((size_t)fs.base[6]) : nullptr;
        double* fud = lg.nest ? c.take<double>((size_t)fs.ebase[6]) : nullptr;
        if (L) {
          L->d.u[0] = u0d;
          L->d.u[1] = nullptr;
          L->d.inter = ind;
          L->d.fc_unc = fud;
        }
      }
    }
    if (leaf) {
      double* f = c.take<double>(e);
      if (L) {
        L->f = f;
        L->nblocks = norm_blocks(G);
        L->partial_off = slots;
      }
      slots += norm_blocks(G);
      const long long dense = (long long)lg.n[0] * lg.n[1] * lg.n[2];
      if (L) L->stage_off = 4 * leaf_total;
      leaf_total += dense;
      if (dense > max_leaf) max_leaf = dense;
      if ((long long)e > max_leaf_padded) max_leaf_padded = (long long)e;
    }
    if (l == 0) {
      double* k = c.take<double>((size_t)lg.n[0] * lg.n[1] * lg.n[2]);
      if (L) L->kern = k;
    }
  }
  double* partial = c.take<double>((size_t)slots * 2);
  double* red = c.take<double>(kRedDoubles);
  double* scratch = c.take<double>((size_t)3 * max_leaf);
  double* tau_work = c.take<double>((size_t)3 * max_leaf_padded);
  double* stage = c.take<double>((size_t)4 * leaf_total);
  if (h) {
    h->tau_work = tau_work;
    h->stage = stage;
    h->partial_slots = slots;
    h->partial = partial;
    h->red = red;
    h->wait_err = reinterpret_cast<unsigned*>(red + 4);
    h->scratch = scratch;
    h->scratch_elems = max_leaf;
  }
  return c.used;
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
  if (cfg->precision == MG_MIXED && (cfg->inner_cycles < 1 || cfg->inner_cycles > 16)) {
    if (msg && len) snprintf(msg, len, "inner_cycles must be in [1, 16] for MG_MIXED");
    return false;
  }
  if (cfg->nu1 < 0 || cfg->nu2 < 0 || cfg->nu1 + cfg->nu2 < 1 || cfg->nu1 > 16 || cfg->nu2 > 16) {
    if (msg && len) snprintf(msg, len, "nu1, nu2 must be in [0, 16] with nu1 + nu2 >= 1");
    return false;
  }
  if (cfg->tile_rows < 0 || cfg->tile_rows > 8) {
    if (msg && len) snprintf(msg, len, "tile_rows must be in [0, 8]");
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
  p.bytes = carve(cfg, p, nullptr, nullptr);
  if (plan) *plan = p;
  return true;
}

int finest(const mg_hierarchy* h) { return (int)h->L.size() - 1; }

// Levels smoothed by the TMA-staged kernel by default: float32 nests of >= 2^23
// cells.  Measured in CUDA graphs on GB300: it beats the plain kernel by ~25% on a
// 256^3 float32 nest, ties at 128^3 and loses below (each block marches through 8
// planes in sequence, so small grids have too few blocks), and loses on periodic
// levels (ghost-image stores); the float64 smoother is bound by the FP64 pipe.
constexpr long long kTmaMinCells = 1ll << 23;

template <typename T>
cudaError_t setup_tma_bufs(const mg_hierarchy* h, DevLevel& L, Bufs<T>& b) {
  const int fl = h->cfg.flags;
  b.tma = false;
  if (fl & MG_FLAG_NO_TMA) return cudaSuccess;
  if (!(fl & MG_FLAG_TMA_ALL) &&
      (sizeof(T) != 4 || L.periodic || cells_of(L.G) < kTmaMinCells))
    return cudaSuccess;
  if (!b.u[0] || !b.u[1] || !b.ffas || !smooth_tma_usable(L.G)) return cudaSuccess;
  for (int q = 0; q < 2; ++q) {
    const cudaError_t e =
        make_plane_tmap(L.G, b.u[q], (int)sizeof(T), h->cfg.order, true, &b.tm[q]);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = make_plane_tmap(L.G, b.ffas, (int)sizeof(T), h->cfg.order, false, &b.tm_f);
  if (e != cudaSuccess) return e;
  b.tma = true;
  return cudaSuccess;
}

cudaError_t setup_tma(mg_hierarchy* h) {
  if (h->cfg.flags & MG_FLAG_NO_TMA) return cudaSuccess;
  cudaError_t e = prepare_smooth_tma();
  for (DevLevel& L : h->L) {
    if (e != cudaSuccess) break;
    e = h->mixed ? setup_tma_bufs<float>(h, L, L.s) : setup_tma_bufs<double>(h, L, L.d);
  }
  return e;
}
int n_leaf(const mg_hierarchy* h) { return (int)h->L.size() - h->base; }

// ---- level operations, templated on the V-cycle precision --------------------

template <typename T>
mg_status tangential(mg_hierarchy* h, int l) {
  DevLevel& L = h->L[l];
  DevLevel& P = h->L[l - 1];
  Bufs<T>& b = bufs<T>(L);
  Bufs<T>& pb = bufs<T>(P);
  if (recording<T>(h)) {
    POp o = pop(P_TANG);
    o.F = L.G;
    o.P = P.G;
    o.in0 = reinterpret_cast<const float*>(pb.u[pb.cur]);
    o.off = L.off;
    o.fs = L.fs;
    o.s[0] = float(1.0 / P.geo.h);
    o.out0 = reinterpret_cast<float*>(b.inter);
    o.out1 = reinterpret_cast<float*>(b.fc_unc);
    rec_push(h, o, ceil_div((h->cfg.order / 2) * L.fs.ebase[6], kPersistThreads));
    return MG_OK;
  }
  KL(MG_K_GHOST, L.fs.base[6],
     launch_cf_tangential<T>(h->cfg.order, L.G, P.G, pb.u[pb.cur], L.off, L.fs, h->w,
                             1.0 / P.geo.h, b.inter, b.fc_unc, h->s));
  return MG_OK;
}

template <typename T>
mg_status ghost_fill(mg_hierarchy* h, int l, bool edges) {
  DevLevel& L = h->L[l];
  Bufs<T>& b = bufs<T>(L);
  if (L.periodic) {
    if (b.ghosts_stale) {
      if (recording<T>(h)) {
        POp o = pop(P_GHOST_PERIODIC);
        o.F = L.G;
        o.out0 = reinterpret_cast<float*>(b.u[b.cur]);
        rec_push(h, o, ceil_div(ghost_shell_count(L.G), kPersistThreads));
      } else {
        KL(MG_K_GHOST, shell_of(L.G), launch_ghost_periodic<T>(L.G, b.u[b.cur], h->s));
      }
    }
    b.ghosts_stale = false;
    return MG_OK;
  }
  DevLevel& P = h->L[l - 1];
  Bufs<T>& pb = bufs<T>(P);
  if (recording<T>(h) && !edges) {
    // the scale factors exactly as launch_cf_flux rounds them
    const double hh = L.geo.h, invh = 1.0 / L.geo.h, invH = 1.0 / P.geo.h;
    POp o = pop(P_CF_FLUX);
    o.F = L.G;
    o.out0 = reinterpret_cast<float*>(b.u[b.cur]);
    o.fs = L.fs;
    o.in0 = reinterpret_cast<const float*>(b.inter);
    o.in1 = reinterpret_cast<const float*>(b.fc_unc);
    o.s[0] = float(0.125 * invH);
    o.s[1] = float(hh / h->w.ghost_coef[0]);
    o.s[2] = float(hh / h->w.ghost_coef[1]);
    o.s[3] = float(0.25 * invh * hh / h->w.ghost_coef[0]);
    o.s[4] = float(0.25 * invh * hh / h->w.ghost_coef[1]);
    rec_push(h, o, ceil_div(4 * L.fs.ebase[6], kPersistThreads));
    return MG_OK;
  }
  KL(MG_K_GHOST, 4 * L.fs.ebase[6] * L.G.g,
     launch_cf_flux<T>(h->cfg.order, L.G, b.u[b.cur], L.fs, h->w, b.inter, b.fc_unc, L.geo.h,
                       1.0 / L.geo.h, 1.0 / P.geo.h, 1, h->s));
  if (edges)
    KL(MG_K_GHOST, shell_of(L.G),
       launch_cf_edges<T>(h->cfg.order, L.G, b.u[b.cur], P.G, pb.u[pb.cur], L.off, h->w, h->s));
  return MG_OK;
}

template <typename T>
mg_status half_sweep(mg_hierarchy* h, int l, int colour) {
  DevLevel& L = h->L[l];
  Bufs<T>& b = bufs<T>(L);
  ST(ghost_fill<T>(h, l, false));
  const double a_f = L.geo.h * L.geo.h / centre_weight(h->cfg.order);
  if (recording<T>(h)) {
    // the plain smoother's arithmetic (bit-identical to the TMA-staged one), 32 x 4
    // threads per block
    POp o = pop(P_SMOOTH);
    o.F = L.G;
    o.in0 = reinterpret_cast<const float*>(b.u[b.cur]);
    o.out0 = reinterpret_cast<float*>(b.u[1 - b.cur]);
    o.in1 = reinterpret_cast<const float*>(b.ffas);
    o.s[0] = float(a_f);
    o.colour = colour;
    o.periodic = L.periodic ? 1 : 0;
    const long long gx = ceil_div((L.G.n2 + 1) / 2, 32), gy = ceil_div(L.G.n1, 4);
    rec_push(h, o, gx * gy * L.G.n0, (int)gx, (int)gy);
    b.cur ^= 1;
    return MG_OK;
  }
  if (b.tma)
    KL(MG_K_SMOOTH, (cells_of(L.G) + 1) / 2,
       launch_smooth_half_tma<T>(h->cfg.order, L.G, &b.tm[b.cur], &b.tm_f, b.u[1 - b.cur], a_f,
                                 colour, L.periodic ? 1 : 0, h->wait_err, h->s));
  else
    KL(MG_K_SMOOTH, (cells_of(L.G) + 1) / 2,
       launch_smooth_half<T>(h->cfg.order, L.G, b.u[b.cur], b.u[1 - b.cur], b.ffas, a_f, colour,
                             L.periodic ? 1 : 0, h->cfg.tile_rows > 0 ? h->cfg.tile_rows : 4,
                             !(h->cfg.flags & MG_FLAG_PAIR_SMOOTHER), h->s));
  b.cur ^= 1;
  return MG_OK;
}

template <typename T>
mg_status smooth(mg_hierarchy* h, int l, int sweeps) {
  for (int s = 0; s < sweeps; ++s) {
    ST(half_sweep<T>(h, l, 0));
    ST(half_sweep<T>(h, l, 1));
  }
  return MG_OK;
}

template <typename T>
mg_status vcycle(mg_hierarchy* h, int l) {
  DevLevel& L = h->L[l];
  Bufs<T>& b = bufs<T>(L);
  const int order = h->cfg.order;
  if (l == 0) {
    if (recording<T>(h)) {
      POp o = pop(P_COARSEST);
      o.F = L.G;
      o.in0 = reinterpret_cast<const float*>(b.ffas);
      o.out0 = reinterpret_cast<float*>(b.u[b.cur]);
      o.kern = L.kern;
      rec_push(h, o, cells_of(L.G));
      return MG_OK;
    }
    KL(MG_K_COARSEST, cells_of(L.G), launch_coarsest(L.G, b.ffas, b.u[b.cur], L.kern, h->s));
    return MG_OK;
  }
  DevLevel& P = h->L[l - 1];
  Bufs<T>& pb = bufs<T>(P);
  ST(smooth<T>(h, l, h->cfg.nu1));
  ST(ghost_fill<T>(h, l, false));
  if (recording<T>(h)) {
    const long long gx = ceil_div(L.cn.z, 32), gy = ceil_div(L.cn.y, 4);
    POp o = pop(P_RESTRICT);
    o.F = L.G;
    o.P = P.G;
    o.in0 = reinterpret_cast<const float*>(b.u[b.cur]);
    o.in1 = reinterpret_cast<const float*>(b.ffas);
    o.s[0] = float(1.0 / (L.geo.h * L.geo.h));
    o.out0 = reinterpret_cast<float*>(pb.u[pb.cur]);
    o.out1 = reinterpret_cast<float*>(pb.ffas);
    o.out2 = reinterpret_cast<float*>(b.ubar);
    o.off = L.off;
    o.cn = L.cn;
    o.periodic = P.periodic ? 1 : 0;
    rec_push(h, o, gx * gy * L.cn.x, (int)gx, (int)gy);
    POp q = pop(P_FAS);
    q.P = P.G;
    q.in0 = reinterpret_cast<const float*>(pb.u[pb.cur]);
    q.out0 = reinterpret_cast<float*>(pb.ffas);
    q.s[0] = float(1.0 / (P.geo.h * P.geo.h));
    q.off = L.off;
    q.cn = L.cn;
    rec_push(h, q, gx * gy * L.cn.x, (int)gx, (int)gy);
    ST(vcycle<T>(h, l - 1));
    if (!L.periodic) ST(tangential<T>(h, l));
    const long long px = ceil_div(L.G.n2 / 2, 32), py = ceil_div(L.G.n1, 4);
    POp r = pop(P_PROLONG);
    r.F = L.G;
    r.out0 = reinterpret_cast<float*>(b.u[b.cur]);
    r.P = P.G;
    r.in0 = reinterpret_cast<const float*>(pb.u[pb.cur]);
    r.in1 = reinterpret_cast<const float*>(b.ubar);
    r.off = L.off;
    r.cn = L.cn;
    r.periodic = L.periodic ? 1 : 0;
    rec_push(h, r, px * py * L.G.n0, (int)px, (int)py);
    ST(smooth<T>(h, l, h->cfg.nu2));
    return MG_OK;
  }
  KL(MG_K_RESTRICT, cells_of(L.G),
     launch_residual_restrict<T>(order, L.G, b.u[b.cur], b.ffas, 1.0 / (L.geo.h * L.geo.h), P.G,
                                 pb.u[pb.cur], pb.ffas, b.ubar, L.off, L.cn,
                                 P.periodic ? 1 : 0, h->s));
  KL(MG_K_FAS, cells_of(L.cn),
     launch_fas_source<T>(order, P.G, pb.u[pb.cur], pb.ffas, 1.0 / (P.geo.h * P.geo.h), L.off,
                          L.cn, h->s));
  ST(vcycle<T>(h, l - 1));
  if (!L.periodic) ST(tangential<T>(h, l));
  KL(MG_K_PROLONG, cells_of(L.G),
     launch_prolong<T>(L.G, b.u[b.cur], P.G, pb.u[pb.cur], b.ubar, L.off, L.cn,
                       L.periodic ? 1 : 0, h->s));
  ST(smooth<T>(h, l, h->cfg.nu2));
  return MG_OK;
}

mg_status fill_zero(mg_hierarchy* h, double* p, long long e) {
  KL(MG_K_COPY, e, launch_fill(p, e, 0.0, h->s));
  return MG_OK;
}

template <typename T>
mg_status zero_state(mg_hierarchy* h, int from_level) {
  for (int l = from_level; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    Bufs<T>& b = bufs<T>(L);
    const long long e = grid_elems(L.G);
    for (int q = 0; q < 2; ++q)
      if (b.u[q]) ST(fill_zero(h, b.u[q], e));
    b.cur = 0;
    b.ghosts_stale = false;
  }
  return MG_OK;
}

// ---- float64 leaf state: sync, norms, residual -------------------------------

double* phi_of(DevLevel& L) { return L.d.u[L.d.cur]; }

mg_status sync_covered(mg_hierarchy* h) {
  for (int l = finest(h); l > h->base; --l) {
    DevLevel& L = h->L[l];
    DevLevel& P = h->L[l - 1];
    KL(MG_K_RESTRICT, cells_of(L.G),
       launch_restrict_u<double>(L.G, phi_of(L), P.G, phi_of(P), L.off, L.cn, h->s));
  }
  return MG_OK;
}

// Partial-sum slots of every leaf level (base first).
LevelRanges leaf_ranges(const mg_hierarchy* h) {
  LevelRanges R{};
  R.n = finest(h) - h->base + 1;
  for (int l = h->base; l <= finest(h); ++l) {
    R.off[l - h->base] = h->L[l].partial_off;
    R.cnt[l - h->base] = h->L[l].nblocks;
  }
  return R;
}

// Leaf residual norm after syncing covered cells, queued on the stream (no
// host synchronisation, so it can be captured); ends with the copy of 4
// doubles to pinned host memory.  In MG_MIXED the residual is also stored
// (float32) as the correction source.
mg_status norm_launches(mg_hierarchy* h, bool zero_u = false, bool copy_out = true) {
  if (!zero_u) ST(sync_covered(h));
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    if (!zero_u) ST(ghost_fill<double>(h, l, false));
    KL(MG_K_NORM, cells_of(L.G),
       launch_norm_partial(h->cfg.order, L.G, zero_u ? nullptr : phi_of(L), L.f,
                           1.0 / (L.geo.h * L.geo.h),
                           L.geo.h * L.geo.h * L.geo.h, L.child_lo, L.child_hi,
                           h->partial + 2 * L.partial_off, L.nblocks,
                           h->mixed ? L.s.ffas : nullptr, h->s));
  }
  KL(MG_K_NORM, h->partial_slots,
     launch_reduce_levels(h->partial, h->partial_slots, leaf_ranges(h), h->red, h->red + 8, h->s));
  if (copy_out)
    CK(cudaMemcpyAsync(h->host_red, h->red, kRedDoubles * sizeof(double), cudaMemcpyDeviceToHost,
                       h->s));
  return MG_OK;
}

// Waits for the queued work, reads the norm record and the event pairs of the
// graph just replayed.
mg_status norm_read(mg_hierarchy* h, double* rr, double* ff, double* fsum) {
  CK(cudaStreamSynchronize(h->s));
  if (h->replayed) {
    for (const ProfEv& ev : h->replayed->evs) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev.a, ev.b));
      h->stats.event_ms[ev.fam] += ms;
      h->stats.timed[ev.fam] += 1;
      h->stats.timed_cells[ev.fam] += ev.cells;
    }
    h->replayed = nullptr;
  }
  unsigned flag;
  std::memcpy(&flag, h->host_red + 4, sizeof(flag));
  if (flag)
    return fail(h, MG_ETIMEOUT,
                "a bounded device-side wait ran out (a smoother block's wait for a staged plane "
                "tile, or a persistent batch item's wait for its dependency); outputs are invalid");
  *rr = h->host_red[0];
  *ff = h->host_red[1];
  if (fsum) *fsum = h->host_red[2];
  return MG_OK;
}

void destroy_graph(Graph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  for (ProfEv& ev : g.evs) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  g.evs.clear();
}

// Runs body(h) once: directly, or by replaying the graph captured from it (the
// body's launches depend only on the hierarchy, not on the cycle, because every
// level returns to the same buffer parity after each visit).
// With timed = true the profiled families carry CUDA events; the solve loops
// time the first cycle of every solve, so every level's launches are sampled
// once per solve without event overhead on the other cycles.
template <typename Body>
mg_status run_body(mg_hierarchy* h, bool timed, Body body) {
  const unsigned mask = timed ? h->prof_mask : 0u;
  Graph& g = h->g_cycle[h->mixed ? h->inner_now : 0][timed && mask ? 1 : 0];
  if (h->cfg.flags & MG_FLAG_NO_GRAPHS) {
    const unsigned keep = h->active_mask;
    h->active_mask = mask;
    const mg_status st = body(h);
    h->active_mask = keep;
    return st;
  }
  if (!g.exec || g.mask != mask || (mask && g.min_cells != h->prof_min_cells)) {
    destroy_graph(g);
    const mg_stats snap = h->stats;
    CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeRelaxed));
    h->capturing = &g;
    const unsigned keep = h->active_mask;
    h->active_mask = mask;
    const mg_status st = body(h);
    h->active_mask = keep;
    h->capturing = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->s, &graph);
    for (int f = 0; f < MG_K_FAMILIES; ++f) {
      g.delta.launches[f] = h->stats.launches[f] - snap.launches[f];
      g.delta.cells[f] = h->stats.cells[f] - snap.cells[f];
      g.delta.event_ms[f] = 0.0;
      g.delta.timed[f] = 0;
      g.delta.timed_cells[f] = 0;
    }
    h->stats = snap;
    if (st != MG_OK) {
      if (graph) cudaGraphDestroy(graph);
      destroy_graph(g);
      return st;
    }
    CK(e);
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    g.mask = mask;
    g.min_cells = h->prof_min_cells;
  }
  CK(cudaGraphLaunch(g.exec, h->s));
  for (int f = 0; f < MG_K_FAMILIES; ++f) {
    h->stats.launches[f] += g.delta.launches[f];
    h->stats.cells[f] += g.delta.cells[f];
  }
  h->replayed = &g;
  return MG_OK;
}

mg_status fp64_cycle_body(mg_hierarchy* h) {
  ST(vcycle<double>(h, finest(h)));
  return norm_launches(h);
}

// Correction e = 0 on every level: only the current buffer needs zeros (the
// smoother writes every interior cell and, on periodic levels, every ghost of
// the other buffer before it is read), and a zero parent gives zero
// tangential intermediate values and parent fluxes on every nest.
mg_status zero_correction(mg_hierarchy* h) {
  auto zero = [&](float* p, long long n) -> mg_status {
    if (h->rec) {
      POp o = pop(P_ZERO);
      o.out0 = p;
      o.n = n;
      rec_push(h, o, ceil_div(n, kZeroPerBlock));
      return MG_OK;
    }
    CK(cudaMemsetAsync(p, 0, (size_t)n * sizeof(float), h->s));
    return MG_OK;
  };
  for (int l = 0; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    L.s.cur = 0;
    L.s.ghosts_stale = false;
    ST(zero(L.s.u[0], grid_elems(L.G)));
    if (L.geo.nest) {
      ST(zero(L.s.inter, L.fs.base[6]));
      ST(zero(L.s.fc_unc, L.fs.ebase[6]));
    }
  }
  return MG_OK;
}

// The float32 half of an outer iteration: zero correction, inner_now V-cycles.
mg_status mixed_inner(mg_hierarchy* h) {
  ST(zero_correction(h));
  for (int m = 0; m < h->inner_now; ++m) ST(vcycle<float>(h, finest(h)));
  return MG_OK;
}

// The float64 half: u += e on the leaf levels, the solution's tangential ghosts, the
// leaf residual (the next correction source) and its norm.
mg_status mixed_tail(mg_hierarchy* h) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    KL(MG_K_PROLONG, cells_of(L.G),
       launch_add_correction(L.G, phi_of(L), L.s.u[L.s.cur], L.periodic ? 1 : 0, h->s));
  }
  for (int l = h->base + 1; l <= finest(h); ++l) ST(tangential<double>(h, l));
  return norm_launches(h);
}

mg_status mixed_outer_body(mg_hierarchy* h) {
  ST(mixed_inner(h));
  return mixed_tail(h);
}

// f on the leaf levels holds the source: remove its composite mean.
mg_status remove_source_mean(mg_hierarchy* h) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    KL(MG_K_NORM, cells_of(L.G),
       launch_sum_partial(L.G, L.f, L.geo.h * L.geo.h * L.geo.h, L.child_lo, L.child_hi,
                          h->partial + 2 * L.partial_off, L.nblocks, h->s));
  }
  KL(MG_K_NORM, h->partial_slots,
     launch_reduce_partials(h->partial, h->partial_slots, 2, h->red + 2, h->s));
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    KL(MG_K_COPY, cells_of(L.G),
       launch_shift_copy(L.G, L.f, h->mixed ? nullptr : L.d.ffas, h->red + 2, 1.0 / h->volume,
                         h->s));
  }
  return MG_OK;
}

mg_status finish_info(mg_hierarchy* h, mg_info& local, double rel, bool at_floor,
                      mg_info* info) {
  local.rel_residual = rel;
  if (info) *info = local;
  const bool fixed = !(h->cfg.tol > 0.0);
  if (!std::isfinite(rel)) return fail(h, MG_ENOCONV, "residual is not finite");
  if (!fixed && rel > h->cfg.tol && !at_floor)
    return fail(h, MG_ENOCONV, "max_cycles reached above tol");
  return MG_OK;
}

void record(mg_info& local, double rel) {
  if (local.cycles < MG_MAX_HISTORY) local.history[local.cycles] = rel;
  local.cycles++;
}

// A solve in phases, so that one hierarchy can run alone or as a member of a
// batch whose iterations are replayed together.
struct SolveState {
  mg_info local;
  double rel = INFINITY;
  int c = 0;
  bool done = false;
  bool at_floor = false;  // residual at the rounding level of the source (see below)
};

// Queues the set-up: composite mean removal, zero solution, tangential caches
// and, in MG_MIXED, the first residual (the source itself: u = 0).
mg_status solve_begin(mg_hierarchy* h) {
  ST(remove_source_mean(h));
  ST(zero_state<double>(h, h->mixed ? h->base : 0));
  for (int l = h->base + 1; l <= finest(h); ++l) ST(tangential<double>(h, l));
  if (h->mixed) ST(norm_launches(h, true));
  return MG_OK;
}

mg_status solve_begin_read(mg_hierarchy* h, SolveState& st) {
  std::memset(&st.local, 0, sizeof(st.local));
  st.c = 0;
  st.done = false;
  st.rel = INFINITY;
  if (h->mixed) {
    // with u = 0 the first residual is the source itself (relative norm 1): no host
    // read here; the source mean arrives with the first iteration's norm
    st.rel = 1.0;
    h->inner_now = h->cfg.inner_cycles;
  }
  return MG_OK;
}

// MG_MIXED: float32 V-cycles for the next outer iteration.  The first one runs
// inner_cycles; later ones run just enough cycles to take the float64 residual from
// rel to a quarter of the tolerance, at most inner_cycles (the stopping test stays the
// float64 residual).  The first V-cycle from a zero correction reduces the residual
// much less than the later ones (about 0.3 against 0.08 in float64 histories of the
// nested workloads), so n cycles are taken to reduce it by exp(-(k n - c)), c = ln 5,
// with k fitted to the previous outer iteration.  A plain geometric rate planned
// single cycles that left the residual where it was (deep nests: 1.3e-7 -> 1.7e-7),
// costing a whole further outer iteration.
int next_inner_cycles(const mg_hierarchy* h, double rel_before, double rel_after, int used) {
  return mgloop::inner_plan(h->cfg.inner_cycles, h->cfg.tol, rel_before, rel_after, used);
}

// The launches of one V-cycle (MG_FP64) or one outer iteration (MG_MIXED).
mg_status solve_body(mg_hierarchy* h) {
  return h->mixed ? mixed_outer_body(h) : fp64_cycle_body(h);
}

// Reads the convergence record of the iteration just run.
mg_status solve_step_read(mg_hierarchy* h, SolveState& st) {
  double rr, ff, fs;
  ST(norm_read(h, &rr, &ff, &fs));
  if (st.c == 0) st.local.source_mean = fs / h->volume;
  const double before = st.rel;
  st.rel = ff > 0.0 ? std::sqrt(rr) / std::sqrt(ff) : std::sqrt(rr);
  if (h->mixed) {
    st.local.inner_cycles += h->inner_now;
    h->inner_now = next_inner_cycles(h, before, st.rel, h->inner_now);
  }
  record(st.local, st.rel);
  for (int l = h->base; l <= finest(h); ++l)
    st.local.level_rel_residual[l - h->base] =
        mgloop::level_relative(h->host_red[8 + 2 * (l - h->base)], h->host_red[9 + 2 * (l - h->base)]);
  st.c++;
  const bool fixed = !(h->cfg.tol > 0.0);
  // A source that is constant up to rounding (zero after the mean removal but for
  // its rounding) has no meaningful relative residual: the solve stops once the
  // residual is at the rounding level of the source before the mean removal,
  // 64 eps (|f|^2 + V mean^2)^{1/2} (volume-weighted; the solution is then ~0).
  const double mean = st.local.source_mean;
  const double floor = 64.0 * DBL_EPSILON * std::sqrt(ff + h->volume * mean * mean);
  st.at_floor = !fixed && std::sqrt(rr) <= floor;
  st.done = !std::isfinite(st.rel) || (!fixed && st.rel <= h->cfg.tol) || st.at_floor ||
            st.c >= h->cfg.max_cycles;
  return MG_OK;
}

// The periodic problem fixes u only up to a constant.  The float64 V-cycle
// converges to zero mean over the base level (covered cells holding the mean
// of their children), the gauge its exact coarsest solve sets; the float64
// residual of the mixed-precision refinement does not see constants, so its
// result is shifted to the same gauge.
mg_status gauge_zero_base_mean(mg_hierarchy* h) {
  ST(sync_covered(h));
  DevLevel& B = h->L[h->base];
  const Int3 none{0, 0, 0};
  KL(MG_K_NORM, cells_of(B.G),
     launch_sum_partial(B.G, phi_of(B), 1.0, none, none, h->partial + 2 * B.partial_off,
                        B.nblocks, h->s));
  KL(MG_K_NORM, B.nblocks,
     launch_reduce_partials(h->partial + 2 * B.partial_off, B.nblocks, 2, h->red + 2, h->s));
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    KL(MG_K_COPY, grid_elems(L.G),
       launch_sub_mean(phi_of(L), grid_elems(L.G), h->red + 2, 1.0 / (double)cells_of(B.G),
                       h->s));
  }
  for (int l = h->base + 1; l <= finest(h); ++l) ST(tangential<double>(h, l));
  return MG_OK;
}

mg_status solve_end(mg_hierarchy* h, SolveState& st, mg_info* info) {
  const mg_status res = finish_info(h, st.local, st.rel, st.at_floor, info);
  if (res != MG_OK && res != MG_ENOCONV) return res;
  if (h->mixed) ST(gauge_zero_base_mean(h));
  return res;
}

// ---- device-side iteration loop (MG_FLAG_DEVICE_LOOP) ----------------------------
//
// The whole iteration loop of a solve as one CUDA graph: a while node repeats the
// iteration (MG_FP64: V-cycle + norm; MG_MIXED: a switch node selecting the body
// with the planned number of float32 V-cycles, then the float64 update and norm)
// followed by k_loop_step, which applies the stopping rule and the inner-cycle plan
// of the host loop on the device and sets the conditions for the next pass.  The
// host launches the graph once per solve and reads the record at the end, so no
// host round trip separates two iterations.

bool device_loop_on(const mg_hierarchy* h) {
  return (h->cfg.flags & MG_FLAG_DEVICE_LOOP) && !(h->cfg.flags & MG_FLAG_NO_GRAPHS) &&
         h->prof_mask == 0 && h->cfg.max_cycles >= 1 && h->cfg.inner_cycles <= 16;
}

// Captures body(h) on the hierarchy's stream into graph g (after the nodes in
// deps); the launches are counted into *delta instead of the statistics.
template <typename Body>
mg_status capture_into(mg_hierarchy* h, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                       mg_stats* delta, Body body) {
  const mg_stats snap = h->stats;
  CK(cudaStreamBeginCaptureToGraph(h->s, g, deps, nullptr, ndeps, cudaStreamCaptureModeRelaxed));
  const unsigned keep = h->active_mask;
  h->active_mask = 0;
  const mg_status st = body(h);
  h->active_mask = keep;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->s, &out);
  for (int f = 0; f < MG_K_FAMILIES; ++f) {
    delta->launches[f] = h->stats.launches[f] - snap.launches[f];
    delta->cells[f] = h->stats.cells[f] - snap.cells[f];
  }
  h->stats = snap;
  ST(st);
  CK(e);
  return MG_OK;
}

mg_status build_loop_graph(mg_hierarchy* h) {
  LoopGraph& G = h->loop;
  if (!h->loop_dev) CK(cudaMalloc(&h->loop_dev, sizeof(LoopState)));
  if (!h->loop_host) CK(cudaHostAlloc(&h->loop_host, sizeof(LoopState), cudaHostAllocDefault));
  CK(cudaGraphCreate(&G.graph, 0));
  cudaGraph_t g = G.graph;
  const int cap = h->mixed ? h->cfg.inner_cycles : 0;
  cudaGraphConditionalHandle while_h = 0, switch_h = 0;
  CK(cudaGraphConditionalHandleCreate(&while_h, g, 1u, cudaGraphCondAssignDefault));
  if (h->mixed)
    CK(cudaGraphConditionalHandleCreate(&switch_h, g, (unsigned)(cap - 1), cudaGraphCondAssignDefault));
  // record initialisation
  mg_stats none;
  LoopState* dev = h->loop_dev;
  const int mixed = h->mixed ? 1 : 0;
  ST(capture_into(h, g, nullptr, 0, &none, [&](mg_hierarchy* hh) -> mg_status {
    mgloop::k_loop_init<<<1, 1, 0, hh->s>>>(dev, mixed, cap);
    return cudaGetLastError() == cudaSuccess ? MG_OK : fail(hh, MG_ECUDA, "k_loop_init launch");
  }));
  cudaGraphNode_t init = nullptr;
  size_t n = 1;
  CK(cudaGraphGetNodes(g, &init, &n));
  // the loop
  cudaGraphNodeParams wp = {};
  std::memset(&wp, 0, sizeof(wp));
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = while_h;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t loop = nullptr;
  CK(cudaGraphAddNode(&loop, g, &init, nullptr, 1, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  mgloop::LoopParams lp;
  lp.tol = h->cfg.tol;
  lp.volume = h->volume;
  lp.max_cycles = h->cfg.max_cycles;
  lp.mixed = mixed;
  lp.cap = cap;
  lp.n_leaf = finest(h) - h->base + 1;
  const double* red = h->red;
  auto step = [&](mg_hierarchy* hh) -> mg_status {
    mgloop::k_loop_step<<<1, 1, 0, hh->s>>>(dev, red, lp, while_h, switch_h);
    return cudaGetLastError() == cudaSuccess ? MG_OK : fail(hh, MG_ECUDA, "k_loop_step launch");
  };
  if (!h->mixed) {
    ST(capture_into(h, body, nullptr, 0, &G.body[0], [&](mg_hierarchy* hh) -> mg_status {
      ST(vcycle<double>(hh, finest(hh)));
      ST(norm_launches(hh, false, false));
      return step(hh);
    }));
  } else {
    cudaGraphNodeParams sp = {};
    std::memset(&sp, 0, sizeof(sp));
    sp.type = cudaGraphNodeTypeConditional;
    sp.conditional.handle = switch_h;
    sp.conditional.type = cudaGraphCondTypeSwitch;
    sp.conditional.size = (unsigned)cap;
    cudaGraphNode_t sw = nullptr;
    CK(cudaGraphAddNode(&sw, body, nullptr, nullptr, 0, &sp));
    for (int m = 1; m <= cap; ++m) {
      ST(capture_into(h, sp.conditional.phGraph_out[m - 1], nullptr, 0, &G.body[m],
                      [&](mg_hierarchy* hh) -> mg_status {
                        ST(zero_correction(hh));
                        for (int k = 0; k < m; ++k) ST(vcycle<float>(hh, finest(hh)));
                        return MG_OK;
                      }));
    }
    ST(capture_into(h, body, &sw, 1, &G.tail, [&](mg_hierarchy* hh) -> mg_status {
      for (int l = hh->base; l <= finest(hh); ++l) {
        DevLevel& L = hh->L[l];
        KL(MG_K_PROLONG, cells_of(L.G),
           launch_add_correction(L.G, phi_of(L), L.s.u[L.s.cur], L.periodic ? 1 : 0, hh->s));
      }
      for (int l = hh->base + 1; l <= finest(hh); ++l) ST(tangential<double>(hh, l));
      ST(norm_launches(hh, false, false));
      return step(hh);
    }));
  }
  cudaGraphNode_t copy = nullptr;
  CK(cudaGraphAddMemcpyNode1D(&copy, g, &loop, 1, h->loop_host, h->loop_dev, sizeof(LoopState),
                              cudaMemcpyDeviceToHost));
  CK(cudaGraphInstantiate(&G.exec, g, 0));
  return MG_OK;
}

mg_status ensure_loop_graph(mg_hierarchy* h) {
  if (h->loop.exec) return MG_OK;
  const mg_status st = build_loop_graph(h);
  if (st != MG_OK) {
    if (h->loop.graph) cudaGraphDestroy(h->loop.graph);
    h->loop = LoopGraph();
  }
  return st;
}

// Launches the loop graph (after solve_begin); the record is read by loop_read.
mg_status loop_launch(mg_hierarchy* h) {
  ST(ensure_loop_graph(h));
  CK(cudaGraphLaunch(h->loop.exec, h->s));
  return MG_OK;
}

// The loop graph has finished: its record into st (as the host loop leaves it) and
// its launches into the statistics.
mg_status loop_read(mg_hierarchy* h, SolveState& st, const LoopState* rec = nullptr) {
  const LoopState& R = rec ? *rec : *h->loop_host;
  std::memset(&st.local, 0, sizeof(st.local));
  st.local.cycles = R.c;
  for (int i = 0; i < R.c && i < MG_MAX_HISTORY; ++i) st.local.history[i] = R.history[i];
  st.local.source_mean = R.source_mean;
  st.local.inner_cycles = R.inner_total;
  for (int l = h->base; l <= finest(h); ++l)
    st.local.level_rel_residual[l - h->base] = R.level_rel[l - h->base];
  st.rel = R.rel;
  st.at_floor = R.at_floor != 0;
  st.c = R.c;
  st.done = true;
  for (int i = 0; i < R.c; ++i) {
    const mg_stats& d = h->mixed ? h->loop.body[i < MG_MAX_HISTORY ? R.inner_hist[i]
                                                                   : h->cfg.inner_cycles]
                                 : h->loop.body[0];
    for (int f = 0; f < MG_K_FAMILIES; ++f) {
      h->stats.launches[f] += d.launches[f] + (h->mixed ? h->loop.tail.launches[f] : 0);
      h->stats.cells[f] += d.cells[f] + (h->mixed ? h->loop.tail.cells[f] : 0);
    }
  }
  if (h->mixed) h->inner_now = R.inner_now;
  if (R.timeout)
    return fail(h, MG_ETIMEOUT,
                "a bounded device-side wait ran out (a smoother block's wait for a staged plane "
                "tile, or a persistent batch item's wait for its dependency); outputs are invalid");
  return MG_OK;
}

mg_status solve_prepared(mg_hierarchy* h, mg_info* info) {
  SolveState st;
  ST(solve_begin(h));
  ST(solve_begin_read(h, st));
  if (device_loop_on(h)) {
    ST(loop_launch(h));
    CK(cudaStreamSynchronize(h->s));
    ST(loop_read(h, st));
    return solve_end(h, st, info);
  }
  while (!st.done) {
    ST(run_body(h, st.c == 0, solve_body));
    ST(solve_step_read(h, st));
  }
  return solve_end(h, st, info);
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

// add (device buffers only): dst = interior + add
mg_status store_leaf(mg_hierarchy* h, int l, const double* padded, double* dst, bool host,
                     double add = 0.0) {
  DevLevel& L = h->L[l];
  if (host) {
    cudaMemcpy3DParms p = dense_padded_parms(L, const_cast<double*>(padded), dst, false);
    CK(cudaMemcpy3DAsync(&p, h->s));
  } else {
    KL(MG_K_COPY, cells_of(L.G), launch_unpack(L.G, padded, dst, h->s, add));
  }
  return MG_OK;
}

// phi (dense per leaf level) -> float64 u; covered cells := mean of children.
mg_status load_potential(mg_hierarchy* h, const double* const phi[], bool host) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    ST(load_leaf(h, l, phi[l - h->base], phi_of(L), host));
    L.d.ghosts_stale = true;
  }
  ST(sync_covered(h));
  for (int l = h->base + 1; l <= finest(h); ++l) ST(tangential<double>(h, l));
  return MG_OK;
}

// tau of the potential currently in the float64 u into f of every leaf level.
mg_status tau_into_f(mg_hierarchy* h) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    ST(ghost_fill<double>(h, l, true));
    KL(MG_K_LPT, cells_of(L.G),
       launch_lpt2_source(h->cfg.order, L.G, phi_of(L), 1.0 / (L.geo.h * L.geo.h), L.f,
                          h->tau_work, h->s));
  }
  for (int l = finest(h); l > h->base; --l) {
    DevLevel& L = h->L[l];
    DevLevel& P = h->L[l - 1];
    KL(MG_K_RESTRICT, cells_of(L.G),
       launch_restrict_u<double>(L.G, L.f, P.G, P.f, L.off, L.cn, h->s));
  }
  return MG_OK;
}

// The finest level's psi (3 dense device arrays) += the hybrid correction of the
// level's current source f (Sec. 3.5.2); plans and buffers are made on first use.
mg_status hybrid_into(mg_hierarchy* h, const double* f_dense, double* const psi[3]) {
  DevLevel& L = h->L[finest(h)];
  if (!h->hybrid) {
    CK(hybrid_create(&h->hybrid, L.G.n0, L.G.n1, L.G.n2, L.geo.h, h->cfg.order, !L.periodic));
  }
  CK(hybrid_apply(h->hybrid, f_dense, psi, h->s));
  return MG_OK;
}

// -G phi of the potential in the float64 u; outputs dense, 3 per leaf level.  With
// hybrid (and MG_FLAG_HYBRID), the finest level's psi also gets the hybrid
// correction of the source in f (the source of the potential just solved for).
mg_status gradient_out(mg_hierarchy* h, double* const disp[], bool host, bool hybrid = false) {
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    const int i = l - h->base;
    ST(ghost_fill<double>(h, l, false));
    double* dx = disp[3 * i];
    double* dy = disp[3 * i + 1];
    double* dz = disp[3 * i + 2];
    const long long n = (long long)L.G.n0 * L.G.n1 * L.G.n2;
    const bool hyb = hybrid && l == finest(h) && (h->cfg.flags & MG_FLAG_HYBRID);
    if (hyb && !h->hybrid_f) CK(cudaMalloc(&h->hybrid_f, n * sizeof(double)));
    if (hyb) ST(store_leaf(h, l, L.f, h->hybrid_f, false));
    if (host) {
      if (!dx && !dy && !dz) continue;
      KL(MG_K_LPT, n,
         launch_gradient(h->cfg.order, L.G, phi_of(L), 1.0 / L.geo.h, h->scratch,
                         h->scratch + n, h->scratch + 2 * n, h->s));
      if (hyb) {
        double* const psi[3] = {h->scratch, h->scratch + n, h->scratch + 2 * n};
        ST(hybrid_into(h, h->hybrid_f, psi));
      }
      for (int a = 0; a < 3; ++a)
        if (disp[3 * i + a])
          CK(cudaMemcpyAsync(disp[3 * i + a], h->scratch + a * n, n * sizeof(double),
                             cudaMemcpyDeviceToHost, h->s));
    } else {
      if (!dx || !dy || !dz) return fail(h, MG_EINVAL, "displacement output pointer is NULL");
      KL(MG_K_LPT, n, launch_gradient(h->cfg.order, L.G, phi_of(L), 1.0 / L.geo.h, dx, dy, dz, h->s));
      if (hyb) {
        double* const psi[3] = {dx, dy, dz};
        ST(hybrid_into(h, h->hybrid_f, psi));
      }
    }
  }
  return MG_OK;
}

// Host-buffer pipelines: phi and the displacements of the solve just finished go
// into the stage (dense, on the device) and their copies to the caller's host
// buffers are queued on the copy stream, where they run while the work stream goes
// on with tau and the second solve (the host link, ~190 GB/s, would otherwise add
// the copies to the step).
mg_status stage_outputs(mg_hierarchy* h, double* const phi[], double* const disp[]) {
  if (!phi && !disp) return MG_OK;
  std::vector<double*> dd;
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    const long long n = cells_of(L.G);
    double* base = h->stage + L.stage_off;
    if (phi && phi[l - h->base]) ST(store_leaf(h, l, phi_of(L), base, false));
    for (int a = 1; a <= 3; ++a) dd.push_back(base + a * n);
  }
  if (disp) ST(gradient_out(h, dd.data(), false, true));
  CK(cudaEventRecord(h->ev_staged, h->s));
  CK(cudaStreamWaitEvent(h->cs, h->ev_staged, 0));
  h->copies_pending = true;
  for (int l = h->base; l <= finest(h); ++l) {
    DevLevel& L = h->L[l];
    const int i = l - h->base;
    const long long n = cells_of(L.G);
    const double* base = h->stage + L.stage_off;
    if (phi && phi[i])
      CK(cudaMemcpyAsync(phi[i], base, n * sizeof(double), cudaMemcpyDeviceToHost, h->cs));
    for (int a = 0; disp && a < 3; ++a)
      if (disp[3 * i + a])
        CK(cudaMemcpyAsync(disp[3 * i + a], base + (a + 1) * n, n * sizeof(double),
                           cudaMemcpyDeviceToHost, h->cs));
  }
  CK(cudaEventRecord(h->ev_copied, h->cs));
  return MG_OK;
}

// Orders the work stream after the staged copies: before the stage is written
// again and before the caller is told that the results are in host memory.
mg_status join_copies(mg_hierarchy* h) {
  if (!h->copies_pending) return MG_OK;
  h->copies_pending = false;
  const cudaError_t e = cudaStreamWaitEvent(h->s, h->ev_copied, 0);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(h->cs);  // no copy may outlive the call
    return fail_cuda(h, e, "cudaStreamWaitEvent(copies)");
  }
  return MG_OK;
}

// Orders the hierarchy's work stream after the caller's stream, runs f, then
// orders the caller's stream after the work.
template <typename F>
mg_status on_streams(mg_hierarchy* h, F f) {
  CK(cudaEventRecord(h->ev_in, h->user_s));
  CK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  const mg_status st = f();
  CK(cudaEventRecord(h->ev_out, h->s));
  CK(cudaStreamWaitEvent(h->user_s, h->ev_out, 0));
  return st;
}

bool check_ptrs(const void* const* p, int count) {
  if (!p) return false;
  for (int i = 0; i < count; ++i)
    if (!p[i]) return false;
  return true;
}

}  // namespace

// ---- batches ---------------------------------------------------------------------
//
// A batch solves independent hierarchies together.  Each member keeps its own
// work stream; the V-cycles (or outer iterations) of all members that have not
// converged yet are captured fork-join into one CUDA graph, one branch per
// member, and replayed with one launch per iteration, so the small kernels of
// different hierarchies run concurrently.  A member leaves the graph once it
// has converged; graphs are cached per set of active members.

namespace {

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<mg_stats> delta;  // launch counts each member adds per replay
  // persistent mode: the work list, member weights and launch state (one allocation)
  void* dbuf = nullptr;
  long long items = 0;  // work items per replay
  int ops = 0;          // level operations per replay
};

}  // namespace

struct mg_batch {
  std::vector<mg_hierarchy*> m;
  cudaStream_t user_s = nullptr;
  cudaStream_t s = nullptr;  // capture / replay stream
  cudaEvent_t ev_in = nullptr, fork = nullptr;
  std::vector<cudaEvent_t> join;   // recorded inside captures only
  std::vector<cudaEvent_t> ready;  // member stream -> batch stream ordering before a replay
  // per set of active members and their bodies: 0 inactive, else 1 + inner cycles
  std::map<std::vector<int>, BatchGraph> graphs;
  int persist_blocks_per_sm = 0;  // persistent launch: blocks per SM (0: as many as fit)
  std::string err;
};

namespace {

mg_status bfail(mg_batch* b, mg_status st, const std::string& msg) {
  b->err = msg;
  return st;
}

#define BCK(expr)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return bfail(b, MG_ECUDA, std::string("CUDA error ") + cudaGetErrorString(e_) + \
                                    " in " #expr);                                 \
  } while (0)

mg_status member_status(mg_batch* b, int i, mg_status st) {
  if (st != MG_OK && st != MG_ENOCONV)
    b->err = "member " + std::to_string(i) + ": " + b->m[i]->err;
  return st;
}

// A member whose float32 V-cycles join the persistent launch: MG_MIXED with
// MG_FLAG_PERSISTENT and graphs on.
bool member_persistent(const mg_hierarchy* h) {
  return h->mixed && (h->cfg.flags & MG_FLAG_PERSISTENT) && !(h->cfg.flags & MG_FLAG_NO_GRAPHS);
}

bool batch_persistent(const mg_batch* b, const std::vector<int>& active) {
  for (size_t i = 0; i < b->m.size(); ++i)
    if (active[i] && member_persistent(b->m[i])) return true;
  return false;
}

constexpr unsigned long long kPersistWaitNs = 2000000000ull;  // 2 s per dependency wait

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Persistent mode: the float32 halves of the active members that set MG_FLAG_PERSISTENT
// are recorded as work lists (the members' host state advances as for a capture),
// uploaded, and captured as [reset state, persistent launch, wait flags] followed by
// each such member's float64 half on its own stream; the other active members' whole
// iterations are captured as branches that run concurrently with the persistent launch.
mg_status batch_graph_persistent(mg_batch* b, const std::vector<int>& active, BatchGraph& g) {
  const size_t n = b->m.size();
  std::vector<int> pers(n, 0), plain(n, 0);
  for (size_t i = 0; i < n; ++i) {
    pers[i] = active[i] && member_persistent(b->m[i]);
    plain[i] = active[i] && !pers[i];
  }
  std::vector<std::vector<POp>> lists(n);
  for (size_t i = 0; i < n; ++i) {
    if (!pers[i]) continue;
    mg_hierarchy* h = b->m[i];
    h->rec = &lists[i];
    const mg_status st = mixed_inner(h);
    h->rec = nullptr;
    if (st != MG_OK) return member_status(b, (int)i, st);
  }
  // member-major work list: member i's chain at ops[mop0[i] .. mop0[i] + mops[i]), its
  // items numbered along the chain
  std::vector<POp> ops;
  std::vector<int> mop0(n, 0), mops(n, 0);
  long long total = 0;
  int active_n = 0;
  for (size_t i = 0; i < n; ++i) {
    mop0[i] = (int)ops.size();
    if (!pers[i]) continue;
    ++active_n;
    long long t = 0;
    for (size_t q = 0; q < lists[i].size(); ++q) {
      POp o = lists[i][q];
      o.member = (int)i;
      o.seq = (int)q;
      o.tile0 = t;
      t += o.ntiles;
      ops.push_back(o);
    }
    if (t > (1ll << 30)) return bfail(b, MG_EINVAL, "persistent batch: work list too long");
    mops[i] = (int)lists[i].size();
    total += t;
  }
  if (ops.empty() || active_n == 0) return bfail(b, MG_EINVAL, "persistent batch: empty work list");
  const size_t wb = persist_weight_bytes();
  const size_t off_w = align_up(ops.size() * sizeof(POp), 256);
  const size_t off_f = align_up(off_w + n * wb, 256);                  // member wait flags
  const size_t off_m = align_up(off_f + n * sizeof(unsigned*), 256);   // mop0[n], mops[n]
  const size_t off_s = align_up(off_m + 2 * n * sizeof(int), 256);     // PState
  const size_t off_d = off_s + align_up(sizeof(PState), 16);           // done[n]
  const size_t off_t = off_d + align_up(n * sizeof(int), 16);          // taken[ops]
  const size_t off_c = off_t + align_up(ops.size() * sizeof(int), 16); // count[ops]
  const size_t bytes = off_c + ops.size() * sizeof(int);
  std::vector<unsigned char> host(off_s, 0);
  std::memcpy(host.data(), ops.data(), ops.size() * sizeof(POp));
  std::vector<unsigned*> flags(n, nullptr);
  for (size_t i = 0; i < n; ++i) {
    persist_weights(b->m[i]->w, host.data() + off_w + i * wb);
    flags[i] = pers[i] ? b->m[i]->wait_err : nullptr;
  }
  std::memcpy(host.data() + off_f, flags.data(), n * sizeof(unsigned*));
  std::memcpy(host.data() + off_m, mop0.data(), n * sizeof(int));
  std::memcpy(host.data() + off_m + n * sizeof(int), mops.data(), n * sizeof(int));
  int grid = 0;
  BCK(persist_grid(&grid));
  if (b->persist_blocks_per_sm > 0) {
    int dev = 0, sms = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    grid = std::min(grid, sms * b->persist_blocks_per_sm);
  }
  char* d = nullptr;
  BCK(cudaMalloc(&d, bytes));
  g.dbuf = d;
  g.items = total;
  g.ops = (int)ops.size();
  BCK(cudaMemcpy(d, host.data(), off_s, cudaMemcpyHostToDevice));
  PState* st = reinterpret_cast<PState*>(d + off_s);
  int* done = reinterpret_cast<int*>(d + off_d);
  int* taken = reinterpret_cast<int*>(d + off_t);
  int* count = reinterpret_cast<int*>(d + off_c);
  const int* dmop0 = reinterpret_cast<const int*>(d + off_m);

  BCK(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeRelaxed));
  mg_status rs = MG_OK;
  cudaError_t e = cudaSuccess;
  // the members outside the persistent launch: their whole iterations as branches
  bool any_plain = false;
  for (size_t i = 0; i < n; ++i) any_plain = any_plain || plain[i];
  if (any_plain) e = cudaEventRecord(b->fork, b->s);
  for (size_t i = 0; i < n && rs == MG_OK && e == cudaSuccess; ++i) {
    if (!plain[i]) continue;
    mg_hierarchy* h = b->m[i];
    e = cudaStreamWaitEvent(h->s, b->fork, 0);
    if (e != cudaSuccess) break;
    const mg_stats snap = h->stats;
    const unsigned keep = h->active_mask;
    h->active_mask = 0;
    rs = solve_body(h);
    h->active_mask = keep;
    for (int f = 0; f < MG_K_FAMILIES; ++f) {
      g.delta[i].launches[f] = h->stats.launches[f] - snap.launches[f];
      g.delta[i].cells[f] = h->stats.cells[f] - snap.cells[f];
    }
    h->stats = snap;
    if (rs != MG_OK) member_status(b, (int)i, rs);
  }
  if (e == cudaSuccess && rs == MG_OK) e = cudaMemsetAsync(d + off_s, 0, bytes - off_s, b->s);
  if (e == cudaSuccess)
    e = launch_persist(reinterpret_cast<const POp*>(d), dmop0, dmop0 + n, (int)n, active_n,
                       d + off_w, st, done, taken, count, kPersistWaitNs, grid, b->s);
  if (e == cudaSuccess)
    e = launch_persist_flags(st, reinterpret_cast<unsigned* const*>(d + off_f), (int)n, b->s);
  if (e == cudaSuccess && rs == MG_OK) e = cudaEventRecord(b->fork, b->s);
  for (size_t i = 0; i < n && rs == MG_OK && e == cudaSuccess; ++i) {
    if (!pers[i]) continue;
    mg_hierarchy* h = b->m[i];
    e = cudaStreamWaitEvent(h->s, b->fork, 0);
    if (e != cudaSuccess) break;
    const mg_stats snap = h->stats;
    const unsigned keep = h->active_mask;
    h->active_mask = 0;
    rs = mixed_tail(h);
    h->active_mask = keep;
    for (int f = 0; f < MG_K_FAMILIES; ++f) {
      g.delta[i].launches[f] = h->stats.launches[f] - snap.launches[f];
      g.delta[i].cells[f] = h->stats.cells[f] - snap.cells[f];
    }
    h->stats = snap;
    if (rs != MG_OK) {
      member_status(b, (int)i, rs);
      break;
    }
    e = cudaEventRecord(b->join[i], h->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s, b->join[i], 0);
  }
  for (size_t i = 0; i < n && rs == MG_OK && e == cudaSuccess; ++i) {
    if (!plain[i]) continue;
    e = cudaEventRecord(b->join[i], b->m[i]->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s, b->join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->s, &graph);
  if (rs != MG_OK || e != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (rs != MG_OK) return rs;
    BCK(e != cudaSuccess ? e : ee);
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  BCK(ei);
  return MG_OK;
}

mg_status batch_graph(mg_batch* b, const std::vector<int>& active, BatchGraph** out) {
  auto it = b->graphs.find(active);
  if (it != b->graphs.end()) {
    *out = &it->second;
    return MG_OK;
  }
  if (batch_persistent(b, active)) {
    BatchGraph g;
    g.delta.resize(b->m.size());
    const mg_status st = batch_graph_persistent(b, active, g);
    if (st != MG_OK) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.dbuf) cudaFree(g.dbuf);
      return st;
    }
    auto res = b->graphs.emplace(active, g);
    *out = &res.first->second;
    return MG_OK;
  }
  BatchGraph g;
  g.delta.resize(b->m.size());
  BCK(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeRelaxed));
  mg_status st = MG_OK;
  cudaError_t e = cudaEventRecord(b->fork, b->s);
  for (size_t i = 0; i < b->m.size() && st == MG_OK && e == cudaSuccess; ++i) {
    if (!active[i]) continue;
    mg_hierarchy* h = b->m[i];
    e = cudaStreamWaitEvent(h->s, b->fork, 0);
    if (e != cudaSuccess) break;
    const mg_stats snap = h->stats;
    const unsigned keep = h->active_mask;
    h->active_mask = 0;
    st = solve_body(h);
    h->active_mask = keep;
    for (int f = 0; f < MG_K_FAMILIES; ++f) {
      g.delta[i].launches[f] = h->stats.launches[f] - snap.launches[f];
      g.delta[i].cells[f] = h->stats.cells[f] - snap.cells[f];
    }
    h->stats = snap;
    if (st != MG_OK) {
      member_status(b, (int)i, st);
      break;
    }
    e = cudaEventRecord(b->join[i], h->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s, b->join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->s, &graph);
  if (st != MG_OK || e != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (st != MG_OK) return st;
    BCK(e != cudaSuccess ? e : ee);
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  BCK(ei);
  auto res = b->graphs.emplace(active, g);
  *out = &res.first->second;
  return MG_OK;
}

// Members with the device-side loop: each member's loop graph on its own stream,
// all launched before the first wait, so the members run concurrently and each one
// stops on its own.
mg_status batch_solve_device_loops(mg_batch* b, mg_info* infos) {
  const size_t n = b->m.size();
  std::vector<SolveState> st(n);
  for (size_t i = 0; i < n; ++i) {
    mg_hierarchy* h = b->m[i];
    mg_status r = solve_begin(h);
    if (r == MG_OK) r = solve_begin_read(h, st[i]);
    if (r == MG_OK) r = loop_launch(h);
    if (r != MG_OK) return member_status(b, (int)i, r);
  }
  mg_status worst = MG_OK;
  for (size_t i = 0; i < n; ++i) {
    mg_hierarchy* h = b->m[i];
    BCK(cudaStreamSynchronize(h->s));
    mg_status r = loop_read(h, st[i]);
    if (r == MG_OK || r == MG_ENOCONV) r = solve_end(h, st[i], infos ? &infos[i] : nullptr);
    if (r != MG_OK && r != MG_ENOCONV) return member_status(b, (int)i, r);
    if (r == MG_ENOCONV) worst = MG_ENOCONV;
  }
  return worst;
}

// Solves every member; f of every member holds its source.
mg_status batch_solve(mg_batch* b, mg_info* infos) {
  const size_t n = b->m.size();
  bool loops = true;
  for (size_t i = 0; i < n; ++i) loops = loops && device_loop_on(b->m[i]);
  if (loops) return batch_solve_device_loops(b, infos);
  std::vector<SolveState> st(n);
  for (size_t i = 0; i < n; ++i) {
    mg_status r = solve_begin(b->m[i]);
    if (r != MG_OK) return member_status(b, (int)i, r);
  }
  for (size_t i = 0; i < n; ++i) {
    mg_status r = solve_begin_read(b->m[i], st[i]);
    if (r != MG_OK) return member_status(b, (int)i, r);
  }
  for (;;) {
    std::vector<int> active(n);
    bool any = false;
    for (size_t i = 0; i < n; ++i) {
      active[i] = st[i].done ? 0 : 1 + (b->m[i]->mixed ? b->m[i]->inner_now : 0);
      any = any || active[i];
    }
    if (!any) break;
    BatchGraph* g = nullptr;
    ST(batch_graph(b, active, &g));
    // the replay runs on the batch stream: order it after everything already
    // queued on the active members' own streams (set-up, tau, previous work)
    for (size_t i = 0; i < n; ++i) {
      if (!active[i]) continue;
      BCK(cudaEventRecord(b->ready[i], b->m[i]->s));
      BCK(cudaStreamWaitEvent(b->s, b->ready[i], 0));
    }
    BCK(cudaGraphLaunch(g->exec, b->s));
    BCK(cudaStreamSynchronize(b->s));
    for (size_t i = 0; i < n; ++i) {
      if (!active[i]) continue;
      mg_hierarchy* h = b->m[i];
      for (int f = 0; f < MG_K_FAMILIES; ++f) {
        h->stats.launches[f] += g->delta[i].launches[f];
        h->stats.cells[f] += g->delta[i].cells[f];
      }
      h->replayed = nullptr;
      mg_status r = solve_step_read(h, st[i]);
      if (r != MG_OK) return member_status(b, (int)i, r);
    }
  }
  mg_status worst = MG_OK;
  for (size_t i = 0; i < n; ++i) {
    mg_status r = solve_end(b->m[i], st[i], infos ? &infos[i] : nullptr);
    if (r != MG_OK && r != MG_ENOCONV) return member_status(b, (int)i, r);
    if (r == MG_ENOCONV) worst = MG_ENOCONV;
  }
  return worst;
}

mg_status batch_pipeline(mg_batch* b, bool host, const double* const* const delta[],
                         double* const* const phi1[], double* const* const phi2[],
                         double* const* const disp1[], double* const* const disp2[],
                         mg_info* info1, mg_info* info2) {
  const size_t n = b->m.size();
  for (size_t i = 0; i < n; ++i) {
    mg_hierarchy* h = b->m[i];
    for (int l = h->base; l <= finest(h); ++l) {
      mg_status r = load_leaf(h, l, delta[i][l - h->base], h->L[l].f, host);
      if (r != MG_OK) return member_status(b, (int)i, r);
    }
  }
  mg_status st1 = batch_solve(b, info1);
  if (st1 != MG_OK && st1 != MG_ENOCONV) return st1;
  for (size_t i = 0; i < n; ++i) {
    mg_hierarchy* h = b->m[i];
    mg_status r = MG_OK;
    if (host) {
      r = stage_outputs(h, phi1 ? phi1[i] : nullptr, disp1 ? disp1[i] : nullptr);
    } else {
      if (phi1 && phi1[i])
        for (int l = h->base; l <= finest(h) && r == MG_OK; ++l)
          if (phi1[i][l - h->base]) r = store_leaf(h, l, phi_of(h->L[l]), phi1[i][l - h->base], host);
      if (r == MG_OK && disp1 && disp1[i]) r = gradient_out(h, disp1[i], host, true);
    }
    if (r == MG_OK) r = tau_into_f(h);
    if (r != MG_OK) return member_status(b, (int)i, r);
  }
  mg_status st2 = batch_solve(b, info2);
  if (st2 != MG_OK && st2 != MG_ENOCONV) return st2;
  for (size_t i = 0; i < n; ++i) {
    mg_hierarchy* h = b->m[i];
    mg_status r = MG_OK;
    if (phi2 && phi2[i])
      for (int l = h->base; l <= finest(h) && r == MG_OK; ++l)
        if (phi2[i][l - h->base]) r = store_leaf(h, l, phi_of(h->L[l]), phi2[i][l - h->base], host);
    if (r == MG_OK && disp2 && disp2[i]) r = gradient_out(h, disp2[i], host, true);
    if (r != MG_OK) return member_status(b, (int)i, r);
  }
  for (size_t i = 0; i < n; ++i) {
    mg_status r = join_copies(b->m[i]);
    if (r != MG_OK) return member_status(b, (int)i, r);
  }
  for (size_t i = 0; i < n; ++i) BCK(cudaStreamSynchronize(b->m[i]->s));
  return st1 != MG_OK ? st1 : st2;
}

}  // namespace

// ---- the whole pipeline without a host round trip (MG_FLAG_DEVICE_LOOP) ----------
//
// With both solves' iteration loops on the device nothing in mg_lpt_pipeline needs a
// value on the host before the end: the loads, the first loop graph, a copy of its
// record, the first outputs, tau, the second loop graph and the second outputs are
// all queued at once and the host waits once.  The records are read afterwards.

namespace {

mg_status pipeline_device_loops(mg_hierarchy* h, bool host, const double* const delta[],
                                double* const phi1[], double* const phi2[],
                                double* const disp1[], double* const disp2[], mg_info* info1,
                                mg_info* info2) {
  if (!h->loop_host1)
    CK(cudaHostAlloc(&h->loop_host1, sizeof(LoopState), cudaHostAllocDefault));
  for (int l = h->base; l <= finest(h); ++l)
    ST(load_leaf(h, l, delta[l - h->base], h->L[l].f, host));
  SolveState st1, st2;
  ST(solve_begin(h));
  ST(solve_begin_read(h, st1));
  ST(loop_launch(h));
  CK(cudaMemcpyAsync(h->loop_host1, h->loop_dev, sizeof(LoopState), cudaMemcpyDeviceToHost, h->s));
  if (h->mixed) ST(gauge_zero_base_mean(h));
  if (host) {
    ST(stage_outputs(h, phi1, disp1));
  } else {
    if (phi1)
      for (int l = h->base; l <= finest(h); ++l)
        if (phi1[l - h->base]) ST(store_leaf(h, l, phi_of(h->L[l]), phi1[l - h->base], false));
    if (disp1) ST(gradient_out(h, disp1, false, true));
  }
  ST(tau_into_f(h));
  ST(solve_begin(h));
  ST(solve_begin_read(h, st2));
  ST(loop_launch(h));
  if (h->mixed) ST(gauge_zero_base_mean(h));
  if (phi2)
    for (int l = h->base; l <= finest(h); ++l)
      if (phi2[l - h->base]) ST(store_leaf(h, l, phi_of(h->L[l]), phi2[l - h->base], host));
  if (disp2) ST(gradient_out(h, disp2, host, true));
  CK(cudaStreamSynchronize(h->s));
  ST(loop_read(h, st1, h->loop_host1));
  const mg_status r1 = finish_info(h, st1.local, st1.rel, st1.at_floor, info1);
  if (r1 != MG_OK && r1 != MG_ENOCONV) return r1;
  ST(loop_read(h, st2));
  const mg_status r2 = finish_info(h, st2.local, st2.rel, st2.at_floor, info2);
  if (r2 != MG_OK && r2 != MG_ENOCONV) return r2;
  return r1 != MG_OK ? r1 : r2;
}

}  // namespace

// ---- non-blocking pipeline jobs (the serving runtime) ---------------------------
//
// mg_lpt_pipeline with host buffers as a state machine that never waits for the
// GPU: job_poll only looks at the event recorded after the work it queued last,
// and once that work has finished it reads the convergence record and queues the
// next piece (the next iteration, the stores and tau between the solves, the
// final stores).  One host thread can so drive the pipelines of many hierarchies,
// each on its own stream, with the same launches as mg_lpt_pipeline.

namespace mgk {

struct PipelineJob {
  mg_hierarchy* h = nullptr;
  std::vector<const double*> delta;
  std::vector<double*> phi1, phi2, disp1, disp2;  // empty: not requested
  int phase = 0;  // 1, 2: solve 1, 2 running; 3: final copies queued; 4: finished
  SolveState st;
  mg_info info[2];
  mg_status res[2] = {MG_OK, MG_OK};
  mg_status status = MG_OK;
  cudaEvent_t ev = nullptr;
};

namespace {

mg_status job_record(PipelineJob* j) {
  mg_hierarchy* h = j->h;
  CK(cudaEventRecord(j->ev, h->s));
  return MG_OK;
}

// Queues the set-up and the first iteration of a solve whose source is in f.
mg_status job_begin_solve(PipelineJob* j) {
  mg_hierarchy* h = j->h;
  ST(solve_begin(h));
  ST(solve_begin_read(h, j->st));
  if (device_loop_on(h))
    ST(loop_launch(h));
  else
    ST(run_body(h, true, solve_body));
  return job_record(j);
}

mg_status job_store(PipelineJob* j, const std::vector<double*>& phi,
                    const std::vector<double*>& disp) {
  mg_hierarchy* h = j->h;
  if (!phi.empty())
    for (int l = h->base; l <= finest(h); ++l)
      ST(store_leaf(h, l, phi_of(h->L[l]), phi[l - h->base], true));
  if (!disp.empty()) ST(gradient_out(h, const_cast<double* const*>(disp.data()), true, true));
  return MG_OK;
}

// The iteration queued last has finished: read it and queue what comes next.
mg_status job_advance(PipelineJob* j) {
  mg_hierarchy* h = j->h;
  if (device_loop_on(h)) {
    ST(loop_read(h, j->st));  // the whole loop of the solve has run
  } else {
    ST(solve_step_read(h, j->st));  // its stream synchronisation returns at once
    if (!j->st.done) {
      ST(run_body(h, false, solve_body));
      return job_record(j);
    }
  }
  const int k = j->phase - 1;
  const mg_status e = solve_end(h, j->st, &j->info[k]);
  if (e != MG_OK && e != MG_ENOCONV) return e;
  j->res[k] = e;
  if (j->phase == 1) {
    ST(stage_outputs(h, j->phi1.empty() ? nullptr : j->phi1.data(),
                     j->disp1.empty() ? nullptr : j->disp1.data()));
    ST(tau_into_f(h));
    j->phase = 2;
    return job_begin_solve(j);
  }
  ST(job_store(j, j->phi2, j->disp2));
  ST(join_copies(h));
  j->phase = 3;
  return job_record(j);
}

void job_finish(PipelineJob* j, mg_status st) {
  if (st != MG_OK) {
    // nothing may still write the caller's buffers once the job reports
    cudaStreamSynchronize(j->h->s);
    cudaStreamSynchronize(j->h->cs);
    j->h->copies_pending = false;
    j->status = st;
  } else {
    j->status = j->res[0] != MG_OK ? j->res[0] : j->res[1];
  }
  j->phase = 4;
}

bool ptr_array(const double* const* p, int count, bool required) {
  if (!p) return !required;
  for (int i = 0; i < count; ++i)
    if (!p[i]) return false;
  return true;
}

}  // namespace

mg_status job_start(mg_hierarchy* h, const double* const delta[], double* const phi1[],
                    double* const phi2[], double* const disp1[], double* const disp2[],
                    PipelineJob** out) {
  *out = nullptr;
  const int nleaf = n_leaf(h);
  if (!ptr_array(delta, nleaf, true) || !ptr_array(phi1, nleaf, false) ||
      !ptr_array(phi2, nleaf, false) || !ptr_array(disp1, 3 * nleaf, false) ||
      !ptr_array(disp2, 3 * nleaf, false))
    return fail(h, MG_EINVAL, "delta needs one pointer per level; each output NULL or full");
  PipelineJob* j = new PipelineJob();
  j->h = h;
  j->delta.assign(delta, delta + nleaf);
  if (phi1) j->phi1.assign(phi1, phi1 + nleaf);
  if (phi2) j->phi2.assign(phi2, phi2 + nleaf);
  if (disp1) j->disp1.assign(disp1, disp1 + 3 * nleaf);
  if (disp2) j->disp2.assign(disp2, disp2 + 3 * nleaf);
  const cudaError_t e = cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete j;
    return fail_cuda(h, e, "cudaEventCreateWithFlags");
  }
  *out = j;
  mg_status st = MG_OK;
  for (int l = h->base; l <= finest(h) && st == MG_OK; ++l)
    st = load_leaf(h, l, j->delta[l - h->base], h->L[l].f, true);
  j->phase = 1;
  if (st == MG_OK) st = job_begin_solve(j);
  if (st != MG_OK) job_finish(j, st);
  return MG_OK;
}

int job_poll(PipelineJob* j) {
  if (j->phase == 4) return 2;
  const cudaError_t q = cudaEventQuery(j->ev);
  if (q == cudaErrorNotReady) return 0;
  if (q != cudaSuccess) {
    job_finish(j, fail_cuda(j->h, q, "cudaEventQuery"));
    return 2;
  }
  if (j->phase == 3) {
    job_finish(j, MG_OK);
    return 2;
  }
  const mg_status st = job_advance(j);
  if (st != MG_OK) {
    job_finish(j, st);
    return 2;
  }
  return 1;
}

mg_status job_result(const PipelineJob* j, mg_info* info1, mg_info* info2) {
  if (info1) *info1 = j->info[0];
  if (info2) *info2 = j->info[1];
  return j->status;
}

const char* job_error(const PipelineJob* j) { return j->h->err.c_str(); }

void job_destroy(PipelineJob* j) {
  if (!j) return;
  if (j->ev) cudaEventDestroy(j->ev);
  delete j;
}

}  // namespace mgk

// ---- C ABI -------------------------------------------------------------------

extern "C" {

mg_status mg_batch_create(mg_hierarchy* const members[], int count, void* cuda_stream,
                          mg_batch** out) {
  if (!out || !members || count < 1 || count > 4096) return MG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!members[i]) return MG_EINVAL;
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return MG_EINVAL;
  }
  mg_batch* b = new mg_batch();
  b->m.assign(members, members + count);
  b->user_s = (cudaStream_t)cuda_stream;
  b->join.assign(count, nullptr);
  b->ready.assign(count, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < count && ok; ++i)
    ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ready[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    mg_batch_destroy(b);
    return MG_ECUDA;
  }
  *out = b;
  return MG_OK;
}

mg_status mg_batch_destroy(mg_batch* b) {
  if (!b) return MG_OK;
  if (b->s) cudaStreamSynchronize(b->s);
  for (auto& kv : b->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.dbuf) cudaFree(kv.second.dbuf);
  }
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ready)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->s) cudaStreamDestroy(b->s);
  delete b;
  return MG_OK;
}

const char* mg_batch_last_error(const mg_batch* b) { return b ? b->err.c_str() : ""; }

mg_status mg_batch_set_persistent_blocks(mg_batch* b, int blocks_per_sm) {
  if (!b || blocks_per_sm < 0 || blocks_per_sm > 64) return MG_EINVAL;
  if (b->persist_blocks_per_sm != blocks_per_sm) {
    if (b->s) cudaStreamSynchronize(b->s);
    for (auto& kv : b->graphs) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      if (kv.second.dbuf) cudaFree(kv.second.dbuf);
    }
    b->graphs.clear();
    b->persist_blocks_per_sm = blocks_per_sm;
  }
  return MG_OK;
}

mg_status mg_batch_lpt_pipeline(mg_batch* b, int host_buffers, const double* const* const delta[],
                                double* const* const phi1[], double* const* const phi2[],
                                double* const* const disp1[], double* const* const disp2[],
                                mg_info* info1, mg_info* info2) {
  if (!b || !delta) return MG_EINVAL;
  const bool host = host_buffers != 0;
  for (size_t i = 0; i < b->m.size(); ++i) {
    mg_hierarchy* h = b->m[i];
    const int nleaf = n_leaf(h);
    if (!check_ptrs((const void* const*)delta[i], nleaf))
      return bfail(b, MG_EINVAL, "member " + std::to_string(i) + ": delta pointers missing");
    if (!host && (!disp1 || !disp2 || !check_ptrs((const void* const*)disp1[i], 3 * nleaf) ||
                  !check_ptrs((const void* const*)disp2[i], 3 * nleaf)))
      return bfail(b, MG_EINVAL, "member " + std::to_string(i) + ": device displacement outputs missing");
  }
  BCK(cudaEventRecord(b->ev_in, b->user_s));
  for (mg_hierarchy* h : b->m) BCK(cudaStreamWaitEvent(h->s, b->ev_in, 0));
  const mg_status st = batch_pipeline(b, host, delta, phi1, phi2, disp1, disp2, info1, info2);
  for (mg_hierarchy* h : b->m) {
    if (h->copies_pending) {  // a failed member left staged copies: let them finish
      cudaStreamSynchronize(h->cs);
      h->copies_pending = false;
    }
    BCK(cudaEventRecord(h->ev_out, h->s));
    BCK(cudaStreamWaitEvent(b->user_s, h->ev_out, 0));
  }
  return st;
}


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
  cfg->inner_cycles = 2;
  cfg->tile_rows = 4;
  cfg->tol = 1e-10;
}

mg_status mg_config_validate(const mg_config* cfg, char* msg, size_t len) {
  if (msg && len) msg[0] = '\0';
  return validate(cfg, msg, len, nullptr) ? MG_OK : MG_EINVAL;
}

size_t mg_workspace_bytes(const mg_config* cfg) {
  Plan p;
  if (!validate(cfg, nullptr, 0, &p)) return 0;
  size_t extra = 0;
  if (cfg->flags & MG_FLAG_HYBRID) {
    const LevelGeom& f = p.geo.back();
    extra = hybrid_bytes(f.n[0], f.n[1], f.n[2], f.nest) +
            (size_t)f.n[0] * f.n[1] * f.n[2] * sizeof(double);
  }
  return p.bytes + extra;
}

int mg_total_levels(const mg_config* cfg) {
  Plan p;
  if (!validate(cfg, nullptr, 0, &p)) return 0;
  return (int)p.geo.size();
}

const char* mg_version(void) { return "mgic-gb300 0.2 (sm_103a)"; }

mg_status mg_set_stream(mg_hierarchy* h, void* cuda_stream) {
  if (!h) return MG_EINVAL;
  h->user_s = (cudaStream_t)cuda_stream;
  return MG_OK;
}

mg_status mg_set_profiling(mg_hierarchy* h, unsigned mask) {
  if (!h) return MG_EINVAL;
  h->prof_mask = mask & ((1u << MG_K_FAMILIES) - 1u);
  h->active_mask = h->prof_mask;
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
      h->stats.timed_cells[f] += h->ev_cells[f][i];
    }
    h->stats.timed[f] += (long long)h->ev_used[f];
    h->ev_used[f] = 0;
  }
  *out = h->stats;
  if (reset) std::memset(&h->stats, 0, sizeof(h->stats));
  return MG_OK;
}

mg_status mg_set_profiling_min_cells(mg_hierarchy* h, long long min_cells) {
  if (!h || min_cells < 0) return MG_EINVAL;
  h->prof_min_cells = min_cells;
  return MG_OK;
}

const char* mg_last_error(const mg_hierarchy* h) { return h ? h->err.c_str() : ""; }

mg_status mg_selftest_wait_limit(void) {
  const Grid G = make_grid(16, 16, 16, 3);
  const size_t e = (size_t)grid_elems(G);
  float *u0 = nullptr, *u1 = nullptr, *f = nullptr;
  unsigned* err = nullptr;
  cudaStream_t s = nullptr;
  mg_status st = MG_OK;
  CUtensorMap t0, tf;
  if (cudaMalloc(&u0, e * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&u1, e * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&f, e * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(unsigned)) != cudaSuccess) {
    st = MG_ENOMEM;
  } else if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
             cudaMemsetAsync(u0, 0, e * sizeof(float), s) != cudaSuccess ||
             cudaMemsetAsync(f, 0, e * sizeof(float), s) != cudaSuccess ||
             cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess ||
             prepare_smooth_tma() != cudaSuccess ||
             make_plane_tmap(G, u0, 4, 6, true, &t0) != cudaSuccess ||
             make_plane_tmap(G, f, 4, 6, false, &tf) != cudaSuccess ||
             launch_smooth_half_tma<float>(6, G, &t0, &tf, u1, 1.0, 0, 1, err, s, 16u) !=
                 cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess) {
    st = MG_ECUDA;
  } else {
    unsigned flag = 0;
    if (cudaMemcpy(&flag, err, sizeof(flag), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = MG_ECUDA;
    else
      st = flag ? MG_ETIMEOUT : MG_OK;
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(u0);
  cudaFree(u1);
  cudaFree(f);
  cudaFree(err);
  return st;
}

mg_status mg_hierarchy_create(const mg_config* cfg, void* cuda_stream, mg_hierarchy** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  Plan plan;
  char msg[256];
  if (!validate(cfg, msg, sizeof(msg), &plan)) return MG_EINVAL;
  mg_hierarchy* h = new mg_hierarchy();
  std::memset(&h->stats, 0, sizeof(h->stats));
  h->cfg = *cfg;
  h->user_s = (cudaStream_t)cuda_stream;
  h->base = plan.base;
  if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_staged, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming) != cudaSuccess) {
    mg_hierarchy_destroy(h);
    return MG_ECUDA;
  }
  h->mixed = cfg->precision == MG_MIXED;
  const int order = cfg->order;
  const int g = order / 2;
  compute_cf_weights(order, &h->w);
  if (cfg->dev_alloc) {
    h->arena = cfg->dev_alloc(plan.bytes, cfg->alloc_ctx);
    if (!h->arena) {
      mg_hierarchy_destroy(h);
      return MG_ENOMEM;
    }
  } else {
    cudaError_t e = cudaMalloc(&h->arena, plan.bytes);
    if (e != cudaSuccess) {
      h->arena = nullptr;
      mg_hierarchy_destroy(h);
      return e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA;
    }
  }
  h->arena_bytes = plan.bytes;
  const size_t nl = plan.geo.size();
  h->L.resize(nl);
  for (size_t l = 0; l < nl; ++l) {
    DevLevel& L = h->L[l];
    L.geo = plan.geo[l];
    L.G = make_grid(L.geo.n[0], L.geo.n[1], L.geo.n[2], g);
    L.periodic = !L.geo.nest;
    L.leaf = (int)l >= h->base;
    L.off = Int3{L.geo.off[0], L.geo.off[1], L.geo.off[2]};
    L.cn = Int3{L.geo.n[0] / 2, L.geo.n[1] / 2, L.geo.n[2] / 2};
    make_faceset(L.G, g, &L.fs);
  }
  carve(cfg, plan, h, (char*)h->arena);
  for (size_t l = 0; l + 1 < nl; ++l) {
    DevLevel& L = h->L[l];
    const DevLevel& C = h->L[l + 1];
    if (L.leaf) {
      L.child_lo = C.off;
      L.child_hi = Int3{C.off.x + C.cn.x, C.off.y + C.cn.y, C.off.z + C.cn.z};
    }
  }
  const LevelGeom& b = plan.geo[plan.base];
  h->volume = b.h * b.h * b.h * (double)b.n[0] * b.n[1] * b.n[2];
  cudaError_t e = cudaMallocHost(&h->host_red, kRedDoubles * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->red, 0, kRedDoubles * sizeof(double), h->s);
  if (e == cudaSuccess) e = setup_tma(h);
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
  for (auto& pair : h->g_cycle) {
    destroy_graph(pair[0]);
    destroy_graph(pair[1]);
  }
  if (h->arena) {
    if (h->cfg.dev_free) h->cfg.dev_free(h->arena, h->cfg.alloc_ctx);
    else cudaFree(h->arena);
  }
  if (h->host_red) cudaFreeHost(h->host_red);
  if (h->loop.exec) cudaGraphExecDestroy(h->loop.exec);
  if (h->loop.graph) cudaGraphDestroy(h->loop.graph);
  cudaFree(h->loop_dev);
  if (h->loop_host) cudaFreeHost(h->loop_host);
  if (h->loop_host1) cudaFreeHost(h->loop_host1);
  hybrid_destroy(h->hybrid);
  cudaFree(h->hybrid_f);
  for (int f = 0; f < MG_K_FAMILIES; ++f) {
    for (cudaEvent_t e : h->ev_start[f]) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_end[f]) cudaEventDestroy(e);
  }
  if (h->cs) cudaStreamSynchronize(h->cs);
  if (h->ev_staged) cudaEventDestroy(h->ev_staged);
  if (h->ev_copied) cudaEventDestroy(h->ev_copied);
  if (h->cs) cudaStreamDestroy(h->cs);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
  return MG_OK;
}

mg_status mg_solve_1lpt(mg_hierarchy* h, const double* const delta[], double* const phi[],
                        mg_info* info) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs((const void* const*)delta, nleaf) || !check_ptrs((const void* const*)phi, nleaf))
    return fail(h, MG_EINVAL, "delta/phi must hold one non-NULL pointer per level");
  return on_streams(h, [&]() -> mg_status {
    for (int l = h->base; l <= finest(h); ++l) ST(load_leaf(h, l, delta[l - h->base], h->L[l].f, false));
    const mg_status st = solve_prepared(h, info);
    if (st != MG_OK && st != MG_ENOCONV) return st;
    for (int l = h->base; l <= finest(h); ++l)
      ST(store_leaf(h, l, phi_of(h->L[l]), phi[l - h->base], false));
    CK(cudaStreamSynchronize(h->s));
    return st;
  });
}

mg_status mg_lpt2_source(mg_hierarchy* h, const double* const phi1[], double* const tau[]) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs((const void* const*)phi1, nleaf) || !check_ptrs((const void* const*)tau, nleaf))
    return fail(h, MG_EINVAL, "phi1/tau must hold one non-NULL pointer per level");
  return on_streams(h, [&]() -> mg_status {
    ST(load_potential(h, phi1, false));
    ST(tau_into_f(h));
    for (int l = h->base; l <= finest(h); ++l) ST(store_leaf(h, l, h->L[l].f, tau[l - h->base], false));
    CK(cudaStreamSynchronize(h->s));
    return MG_OK;
  });
}

mg_status mg_solve_2lpt(mg_hierarchy* h, const double* const phi1[], double* const phi2[],
                        mg_info* info) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs((const void* const*)phi1, nleaf) || !check_ptrs((const void* const*)phi2, nleaf))
    return fail(h, MG_EINVAL, "phi1/phi2 must hold one non-NULL pointer per level");
  return on_streams(h, [&]() -> mg_status {
    ST(load_potential(h, phi1, false));
    ST(tau_into_f(h));
    const mg_status st = solve_prepared(h, info);
    if (st != MG_OK && st != MG_ENOCONV) return st;
    for (int l = h->base; l <= finest(h); ++l)
      ST(store_leaf(h, l, phi_of(h->L[l]), phi2[l - h->base], false));
    CK(cudaStreamSynchronize(h->s));
    return st;
  });
}

mg_status mg_displacements(mg_hierarchy* h, const double* const phi[], double* const disp[]) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs((const void* const*)phi, nleaf) || !check_ptrs((const void* const*)disp, 3 * nleaf))
    return fail(h, MG_EINVAL, "phi/disp must hold 1 and 3 non-NULL pointers per level");
  return on_streams(h, [&]() -> mg_status {
    ST(load_potential(h, phi, false));
    ST(gradient_out(h, disp, false));
    CK(cudaStreamSynchronize(h->s));
    return MG_OK;
  });
}

mg_status mg_hybrid_correction(mg_hierarchy* h, const double* f, double* const psi[3]) {
  if (!h) return MG_EINVAL;
  if (!f || !psi || !psi[0] || !psi[1] || !psi[2])
    return fail(h, MG_EINVAL, "f and the three psi components must be non-NULL");
  return on_streams(h, [&]() -> mg_status {
    ST(hybrid_into(h, f, psi));
    CK(cudaStreamSynchronize(h->s));
    return MG_OK;
  });
}

mg_status mg_lla_density(mg_hierarchy* h, const double* const phi1[], const double* const phi2[],
                         double a1, double a2, double* const rho[]) {
  if (!h) return MG_EINVAL;
  const int nleaf = n_leaf(h);
  if (!check_ptrs((const void* const*)phi1, nleaf) || !check_ptrs((const void* const*)rho, nleaf))
    return fail(h, MG_EINVAL, "phi1/rho must hold one non-NULL pointer per level");
  if (phi2 && !check_ptrs((const void* const*)phi2, nleaf))
    return fail(h, MG_EINVAL, "phi2 must be NULL or hold one non-NULL pointer per level");
  if (!std::isfinite(a1) || !std::isfinite(a2))
    return fail(h, MG_EINVAL, "a1 and a2 must be finite");
  return on_streams(h, [&]() -> mg_status {
    // Phi = a1 phi1 + a2 phi2 into the float64 u of every leaf level
    for (int l = h->base; l <= finest(h); ++l) {
      DevLevel& L = h->L[l];
      const int i = l - h->base;
      KL(MG_K_COPY, cells_of(L.G),
         launch_axpby(cells_of(L.G), a1, phi1[i], a2, phi2 ? phi2[i] : nullptr, h->scratch, h->s));
      ST(load_leaf(h, l, h->scratch, phi_of(L), false));
      L.d.ghosts_stale = true;
    }
    ST(sync_covered(h));
    for (int l = h->base + 1; l <= finest(h); ++l) ST(tangential<double>(h, l));
    // 1/det[I - H] - 1 into f, covered cells := mean of children
    for (int l = h->base; l <= finest(h); ++l) {
      DevLevel& L = h->L[l];
      ST(ghost_fill<double>(h, l, true));
      KL(MG_K_LPT, cells_of(L.G),
         launch_lla(h->cfg.order, L.G, phi_of(L), 1.0 / (L.geo.h * L.geo.h), L.f, h->tau_work,
                    h->s));
    }
    for (int l = finest(h); l > h->base; --l) {
      DevLevel& L = h->L[l];
      DevLevel& P = h->L[l - 1];
      KL(MG_K_RESTRICT, cells_of(L.G),
         launch_restrict_u<double>(L.G, L.f, P.G, P.f, L.off, L.cn, h->s));
    }
    // unit composite mean: remove the volume-weighted leaf mean, then add 1 on output
    ST(remove_source_mean(h));
    for (int l = h->base; l <= finest(h); ++l)
      ST(store_leaf(h, l, h->L[l].f, rho[l - h->base], false, 1.0));
    CK(cudaStreamSynchronize(h->s));
    return MG_OK;
  });
}

mg_status mg_lpt_pipeline(mg_hierarchy* h, int host_buffers, const double* const delta[],
                          double* const phi1[], double* const phi2[], double* const disp1[],
                          double* const disp2[], mg_info* info1, mg_info* info2) {
  if (!h) return MG_EINVAL;
  const bool host = host_buffers != 0;
  const int nleaf = n_leaf(h);
  if (!check_ptrs((const void* const*)delta, nleaf))
    return fail(h, MG_EINVAL, "delta must hold one non-NULL pointer per level");
  if (!host) {
    if (!check_ptrs((const void* const*)disp1, 3 * nleaf) ||
        !check_ptrs((const void* const*)disp2, 3 * nleaf))
      return fail(h, MG_EINVAL, "device displacement outputs must all be set");
  }
  if (device_loop_on(h)) {
    return on_streams(h, [&]() -> mg_status {
      const mg_status st = pipeline_device_loops(h, host, delta, phi1, phi2, disp1, disp2, info1,
                                                 info2);
      const mg_status j = join_copies(h);
      CK(cudaStreamSynchronize(h->s));
      return (st != MG_OK && st != MG_ENOCONV) ? st : (j != MG_OK ? j : st);
    });
  }
  return on_streams(h, [&]() -> mg_status {
    auto steps = [&]() -> mg_status {
      for (int l = h->base; l <= finest(h); ++l)
        ST(load_leaf(h, l, delta[l - h->base], h->L[l].f, host));
      mg_status st1 = solve_prepared(h, info1);
      if (st1 != MG_OK && st1 != MG_ENOCONV) return st1;
      if (host) {
        ST(stage_outputs(h, phi1, disp1));
      } else {
        if (phi1)
          for (int l = h->base; l <= finest(h); ++l)
            if (phi1[l - h->base]) ST(store_leaf(h, l, phi_of(h->L[l]), phi1[l - h->base], host));
        if (disp1) ST(gradient_out(h, disp1, host, true));
      }
      ST(tau_into_f(h));
      mg_status st2 = solve_prepared(h, info2);
      if (st2 != MG_OK && st2 != MG_ENOCONV) return st2;
      if (phi2)
        for (int l = h->base; l <= finest(h); ++l)
          if (phi2[l - h->base]) ST(store_leaf(h, l, phi_of(h->L[l]), phi2[l - h->base], host));
      if (disp2) ST(gradient_out(h, disp2, host, true));
      return st1 != MG_OK ? st1 : st2;
    };
    const mg_status st = steps();
    const mg_status j = join_copies(h);
    CK(cudaStreamSynchronize(h->s));
    return (st != MG_OK && st != MG_ENOCONV) ? st : (j != MG_OK ? j : st);
  });
}

}  // extern "C"
