// Serving runtime (C ABI mg_server_*): a request queue in front of resident
// hierarchies and one native scheduler thread that drives many non-blocking
// pipeline jobs at once.
//
// Each request is the whole initial-conditions step of one hierarchy (1LPT solve,
// 2LPT source and solve, both displacement fields; Sec. 2 and 3 of Hahn & Abel
// 2011) with host buffers in and out.  The scheduler loop:
//   1. admission: pending requests in arrival order; a request takes an idle
//      resident hierarchy of its configuration, or a new one when its
//      mg_workspace_bytes fit the HBM budget after closing idle hierarchies
//      (least recently used first); requests that cannot run yet stay queued;
//   2. progress: for every running job, an event query on the work it queued
//      last; a finished piece is followed at once by the next one (the next
//      V-cycle or outer iteration, tau and the stores between the solves, the
//      final stores), so jobs at different stages overlap on the GPU;
//   3. completion: a finished job's result goes to the result queue and its
//      hierarchy back to the idle cache.
// When nothing moved, the loop yields for ~200 us and then sleeps in 20 us steps
// (yielding throughout while jobs run took a whole core and served no faster).
#include <cuda_runtime.h>
#include <stdint.h>
#include <time.h>

#include <chrono>
#include <atomic>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mg.h"
#include "mg_internal.h"

using namespace mgk;

namespace {

double now_s() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

typedef std::vector<long long> Key;

long long bits_of(double x) {
  long long b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
}

// Every field of the configuration that the hierarchy depends on.
Key config_key(const mg_config& c) {
  Key k = {c.n_levels,
           c.base_n[0],
           c.base_n[1],
           c.base_n[2],
           bits_of(c.box),
           c.order,
           c.precision,
           c.nu1,
           c.nu2,
           c.max_cycles,
           c.inner_cycles,
           c.flags,
           c.tile_rows,
           bits_of(c.tol),
           (long long)(uintptr_t)c.dev_alloc,
           (long long)(uintptr_t)c.dev_free,
           (long long)(uintptr_t)c.alloc_ctx};
  for (int i = 0; i + 1 < c.n_levels && i < MG_MAX_LEVELS - 1; ++i)
    for (int a = 0; a < 3; ++a) {
      k.push_back(c.nest_n[i][a]);
      k.push_back(c.nest_off[i][a]);
    }
  return k;
}

int leaf_levels(const mg_config& c) { return c.n_levels; }

unsigned long long key_hash(const Key& k) {
  unsigned long long x = 1469598103934665603ull;  // FNV-1a over the key's bytes
  for (long long v : k)
    for (int b = 0; b < 8; ++b) {
      x ^= (unsigned long long)((v >> (8 * b)) & 0xff);
      x *= 1099511628211ull;
    }
  return x;
}

struct Slot {
  Key key;
  unsigned long long hash = 0;
  mg_hierarchy* h = nullptr;
  cudaStream_t s = nullptr;
  size_t bytes = 0;
  bool busy = false;
  bool broken = false;  // a CUDA error hit a job on it: closed when released
  unsigned long long last_use = 0;
};

struct Request {
  long long id = 0;
  mg_config cfg;
  Key key;
  unsigned long long hash = 0;
  size_t bytes = 0;
  std::vector<const double*> delta;
  std::vector<double*> phi1, phi2, disp1, disp2;  // empty: not requested
  double t_submit = 0.0, t_start = 0.0;
  Slot* slot = nullptr;
  PipelineJob* job = nullptr;
};

template <typename P>
std::vector<P> copy_ptrs(P const* p, int count) {
  return p ? std::vector<P>(p, p + count) : std::vector<P>();
}

template <typename P>
P* data_or_null(std::vector<P>& v) {
  return v.empty() ? nullptr : v.data();
}

}  // namespace

struct mg_server {
  size_t budget = 0;
  int max_active = 8;
  std::atomic<int> max_instances{0};  // resident hierarchies per configuration (0: no cap)
  int device = 0;
  std::mutex mu;                    // guards everything below up to `th`
  std::condition_variable cv_work;  // a request was queued, or stop
  std::condition_variable cv_done;  // a result was queued
  std::deque<Request*> pending;
  std::deque<mg_server_result> done;
  bool stop = false;
  size_t resident = 0, peak = 0;
  long long created = 0, evictions = 0, completed = 0;
  int n_active = 0, n_slots = 0, peak_active = 0;
  std::thread th;
  // scheduler thread only
  std::vector<Request*> active;
  std::vector<Slot*> slots;
  unsigned long long tick = 0;
  // scheduler accounting (written by the scheduler thread, read by get_stats)
  double t_created = 0.0;
  std::atomic<long long> cpu_ns{0};   // the scheduler thread's CPU time
  std::atomic<long long> busy_ns{0};  // wall time of the passes that moved something
  std::atomic<long long> passes{0};
};

namespace {

void post_result(mg_server* S, Request* r, int status, const mg_info* i1, const mg_info* i2,
                 const char* msg) {
  mg_server_result res;
  std::memset(&res, 0, sizeof(res));
  res.id = r->id;
  res.status = status;
  if (i1) res.info1 = *i1;
  if (i2) res.info2 = *i2;
  res.t_submit = r->t_submit;
  res.t_start = r->t_start;
  res.t_done = now_s();
  if (msg) std::snprintf(res.error, sizeof(res.error), "%s", msg);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.push_back(res);
    S->completed++;
  }
  S->cv_done.notify_all();
  delete r;
}

void close_slot(mg_server* S, Slot* sl) {
  if (sl->h) mg_hierarchy_destroy(sl->h);
  if (sl->s) cudaStreamDestroy(sl->s);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->resident -= sl->bytes;
    S->n_slots--;
  }
  for (size_t i = 0; i < S->slots.size(); ++i)
    if (S->slots[i] == sl) {
      S->slots.erase(S->slots.begin() + (long)i);
      break;
    }
  delete sl;
}

// An idle resident hierarchy of r's configuration, or nullptr.
Slot* find_idle(mg_server* S, const Request* r) {
  for (Slot* sl : S->slots)
    if (!sl->busy && !sl->broken && sl->hash == r->hash && sl->key == r->key) return sl;
  return nullptr;
}

// A new hierarchy for r, after closing idle ones (least recently used first) until
// its bytes fit the budget.  Returns false when r cannot have one now; true with
// *out = nullptr and *msg set when creating it failed.
bool create_for(mg_server* S, Request* r, Slot** out, std::string* msg) {
  *out = nullptr;
  for (;;) {
    size_t resident;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      resident = S->resident;
    }
    if (resident + r->bytes <= S->budget) break;
    Slot* victim = nullptr;
    for (Slot* sl : S->slots)
      if (!sl->busy && (!victim || sl->last_use < victim->last_use)) victim = sl;
    if (!victim) return false;
    close_slot(S, victim);
    std::lock_guard<std::mutex> lk(S->mu);
    S->evictions++;
  }
  Slot* sl = new Slot();
  sl->key = r->key;
  sl->hash = r->hash;
  sl->bytes = r->bytes;
  cudaError_t e = cudaStreamCreateWithFlags(&sl->s, cudaStreamNonBlocking);
  mg_status st = e == cudaSuccess ? mg_hierarchy_create(&r->cfg, sl->s, &sl->h) : MG_ECUDA;
  if (st != MG_OK) {
    *msg = e != cudaSuccess ? std::string("cudaStreamCreate: ") + cudaGetErrorString(e)
                            : std::string("mg_hierarchy_create failed (status ") +
                                  std::to_string((int)st) + ")";
    if (sl->h) mg_hierarchy_destroy(sl->h);
    if (sl->s) cudaStreamDestroy(sl->s);
    delete sl;
    return true;
  }
  S->slots.push_back(sl);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->resident += sl->bytes;
    if (S->resident > S->peak) S->peak = S->resident;
    S->created++;
    S->n_slots++;
  }
  *out = sl;
  return true;
}

void release(mg_server* S, Slot* sl) {
  sl->busy = false;
  sl->last_use = ++S->tick;
  if (sl->broken) close_slot(S, sl);
}

// Starts r on sl (busy from here on); a failure is posted as r's result.
void start_on(mg_server* S, Request* r, Slot* sl) {
  sl->busy = true;
  r->slot = sl;
  r->t_start = now_s();
  const mg_status st = job_start(sl->h, r->delta.data(), data_or_null(r->phi1),
                                 data_or_null(r->phi2), data_or_null(r->disp1),
                                 data_or_null(r->disp2), &r->job);
  if (st != MG_OK) {
    const std::string err = mg_last_error(sl->h);
    release(S, sl);
    post_result(S, r, st, nullptr, nullptr, err.c_str());
    return;
  }
  S->active.push_back(r);
}

// Admission pass; returns whether any request was started or failed.  First every
// pending request (in arrival order, the first kScan) whose configuration has an
// idle resident hierarchy starts on it; then, if there is still room, the oldest
// pending request whose configuration is below the instance cap gets a new
// hierarchy (the others wait for one of theirs to be idle): at most one creation per
// pass, so making
// hierarchies (allocation, and closing idle ones, which waits for the device) never
// holds up the running jobs for long, and a busy configuration gets a second
// hierarchy only when its request is the oldest one waiting.
bool admit(mg_server* S) {
  const size_t kScan = 256;
  std::deque<Request*> cand;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop || S->pending.empty() || (int)S->active.size() >= S->max_active) return false;
    cand.swap(S->pending);
  }
  bool moved = false;
  std::deque<Request*> keep;
  size_t scanned = 0;
  for (Request* r : cand) {
    Slot* sl = nullptr;
    if ((int)S->active.size() < S->max_active && scanned++ < kScan) sl = find_idle(S, r);
    if (sl) {
      start_on(S, r, sl);
      moved = true;
    } else {
      keep.push_back(r);
    }
  }
  // the oldest kept request whose configuration may have one more hierarchy
  auto creatable = keep.end();
  for (auto it = keep.begin(); it != keep.end(); ++it) {
    const int cap = S->max_instances.load(std::memory_order_relaxed);
    if (cap <= 0) {
      creatable = it;
      break;
    }
    int n = 0;
    for (const Slot* sl : S->slots)
      if (sl->hash == (*it)->hash && sl->key == (*it)->key) ++n;
    if (n < cap) {
      creatable = it;
      break;
    }
  }
  if (creatable != keep.end() && (int)S->active.size() < S->max_active) {
    Request* r = *creatable;
    Slot* sl = nullptr;
    std::string msg;
    if (create_for(S, r, &sl, &msg)) {
      keep.erase(creatable);
      moved = true;
      if (sl)
        start_on(S, r, sl);
      else
        post_result(S, r, MG_ECUDA, nullptr, nullptr, msg.c_str());
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  // requests queued meanwhile arrived later: they go behind the ones kept
  S->pending.insert(S->pending.begin(), keep.begin(), keep.end());
  S->n_active = (int)S->active.size();
  if (S->n_active > S->peak_active) S->peak_active = S->n_active;
  return moved;
}

// Progress pass over the running jobs: returns whether any of them moved.
bool advance(mg_server* S) {
  bool moved = false;
  for (size_t i = 0; i < S->active.size();) {
    Request* r = S->active[i];
    const int p = job_poll(r->job);
    if (p == 0) {
      ++i;
      continue;
    }
    moved = true;
    if (p == 1) {
      ++i;
      continue;
    }
    mg_info i1, i2;
    const mg_status st = job_result(r->job, &i1, &i2);
    const std::string msg = (st == MG_OK) ? std::string() : std::string(job_error(r->job));
    job_destroy(r->job);
    r->job = nullptr;
    if (st == MG_ECUDA || st == MG_ETIMEOUT) r->slot->broken = true;
    release(S, r->slot);
    S->active.erase(S->active.begin() + (long)i);
    post_result(S, r, st, &i1, &i2, msg.c_str());
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->n_active = (int)S->active.size();
  return moved;
}

long long thread_cpu_ns() {
  timespec ts;
  clock_gettime(CLOCK_THREAD_CPUTIME_ID, &ts);
  return (long long)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

void scheduler(mg_server* S) {
  cudaSetDevice(S->device);
  double last_move = now_s();
  for (unsigned long long pass = 1;; ++pass) {
    const double t0 = now_s();
    bool moved = admit(S);
    moved = advance(S) || moved;
    S->passes.store((long long)pass, std::memory_order_relaxed);
    if ((pass & 63) == 0) S->cpu_ns.store(thread_cpu_ns(), std::memory_order_relaxed);
    if (moved) {
      last_move = now_s();
      S->busy_ns.fetch_add((long long)(1e9 * (last_move - t0)), std::memory_order_relaxed);
      continue;
    }
    S->cpu_ns.store(thread_cpu_ns(), std::memory_order_relaxed);
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->active.empty()) {
      if (S->stop) break;
      if (S->pending.empty()) {
        S->cv_work.wait(lk, [S] { return S->stop || !S->pending.empty(); });
        last_move = now_s();
        continue;
      }
    }
    lk.unlock();
    if (now_s() - last_move < 200e-6)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

mg_status mg_server_create(unsigned long long hbm_budget, int max_active, mg_server** out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (max_active < 1 || max_active > 256 || hbm_budget == 0) return MG_EINVAL;
  mg_server* S = new mg_server();
  S->budget = (size_t)hbm_budget;
  S->max_active = max_active;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return MG_ECUDA;
  }
  S->t_created = now_s();
  S->th = std::thread(scheduler, S);
  *out = S;
  return MG_OK;
}

mg_status mg_server_set_max_instances(mg_server* S, int n) {
  if (!S || n < 0) return MG_EINVAL;
  S->max_instances.store(n, std::memory_order_relaxed);
  return MG_OK;
}

mg_status mg_server_submit(mg_server* S, long long id, const mg_config* cfg,
                           const double* const delta[], double* const phi1[],
                           double* const phi2[], double* const disp1[], double* const disp2[]) {
  if (!S || !cfg || !delta) return MG_EINVAL;
  if (mg_config_validate(cfg, nullptr, 0) != MG_OK) return MG_EINVAL;
  const size_t bytes = mg_workspace_bytes(cfg);
  if (bytes == 0) return MG_EINVAL;
  if (bytes > S->budget) return MG_ENOMEM;
  const int nleaf = leaf_levels(*cfg);
  for (int i = 0; i < nleaf; ++i)
    if (!delta[i]) return MG_EINVAL;
  Request* r = new Request();
  r->id = id;
  r->cfg = *cfg;
  r->key = config_key(*cfg);
  r->hash = key_hash(r->key);
  r->bytes = bytes;
  r->delta = copy_ptrs(delta, nleaf);
  r->phi1 = copy_ptrs(phi1, nleaf);
  r->phi2 = copy_ptrs(phi2, nleaf);
  r->disp1 = copy_ptrs(disp1, 3 * nleaf);
  r->disp2 = copy_ptrs(disp2, 3 * nleaf);
  for (const auto* v : {&r->phi1, &r->phi2, &r->disp1, &r->disp2})
    for (double* p : *v)
      if (!p) {
        delete r;
        return MG_EINVAL;
      }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete r;
      return MG_EINVAL;
    }
    S->pending.push_back(r);
  }
  S->cv_work.notify_all();
  return MG_OK;
}

int mg_server_poll(mg_server* S, mg_server_result* out, int max, double wait_seconds) {
  if (!S || !out || max < 1) return -1;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_seconds > 0.0)
    S->cv_done.wait_for(lk, std::chrono::duration<double>(wait_seconds),
                        [S] { return !S->done.empty(); });
  int n = 0;
  while (n < max && !S->done.empty()) {
    out[n++] = S->done.front();
    S->done.pop_front();
  }
  return n;
}

mg_status mg_server_get_stats(mg_server* S, mg_server_stats* out) {
  if (!S || !out) return MG_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->resident_bytes = S->resident;
  out->peak_bytes = S->peak;
  out->budget_bytes = S->budget;
  out->created = S->created;
  out->evictions = S->evictions;
  out->completed = S->completed;
  out->pending = (int)S->pending.size();
  out->active = S->n_active;
  out->instances = S->n_slots;
  out->peak_active = S->peak_active;
  out->sched_cpu_s = 1e-9 * (double)S->cpu_ns.load(std::memory_order_relaxed);
  out->sched_busy_s = 1e-9 * (double)S->busy_ns.load(std::memory_order_relaxed);
  out->uptime_s = now_s() - S->t_created;
  out->passes = S->passes.load(std::memory_order_relaxed);
  return MG_OK;
}

mg_status mg_server_destroy(mg_server* S) {
  if (!S) return MG_OK;
  std::deque<Request*> dropped;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    dropped.swap(S->pending);
  }
  S->cv_work.notify_all();
  for (Request* r : dropped) post_result(S, r, MG_EINVAL, nullptr, nullptr, "server closed");
  if (S->th.joinable()) S->th.join();  // the scheduler finishes the running jobs first
  cudaSetDevice(S->device);
  while (!S->slots.empty()) close_slot(S, S->slots.back());
  delete S;
  return MG_OK;
}

}  // extern "C"
