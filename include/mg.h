/*
 * mg.h - C ABI of the GB300 nested-grid Poisson / 2LPT / displacement library.
 *
 * The library solves  L phi = f  (L = finite-difference Laplacian of order 2, 4
 * or 6, Table 1 of Hahn & Abel 2011, arXiv:1103.6031) on a periodic base grid
 * with a chain of nested refinement patches (refinement factor 2, Sec. 3.3) by
 * FAS multigrid V-cycles (Sec. 3.2), computes the second-order LPT source
 * tau = sum_{i<j}(phi_,ii phi_,jj - phi_,ij^2) (Sec. 3.1.2) and the displacement
 * field psi = -grad phi (Sec. 3.1.1).  Every step runs in CUDA kernels on one GPU.
 *
 * Conventions
 *   - Arrays are float64, dense, row-major [nx][ny][nz] (z fastest), one array
 *     per level; level 0 is the periodic base, level i >= 1 is nest i-1.
 *   - A nest of size nest_n (even on every axis, in its own cells) covers the
 *     parent cells [nest_off, nest_off + nest_n/2) on each axis.  Its region must
 *     keep a margin of at least `order` parent cells to the parent's edges.
 *   - Grid spacing h_0 = box / base_n[0]; h_i = h_{i-1} / 2.  The base must be
 *     cubic in spacing (box applies to every axis, h is isotropic).
 *   - phi solves L phi = f - <f>, where <f> is the volume-weighted mean over
 *     leaf cells (cells not covered by a finer level); phi has zero mean over the
 *     base level.  In covered cells the returned phi and f hold the average of
 *     their 8 children.
 *   - psi = -G phi (Table 1 gradient); the caller combines x = q + D1 psi1 +
 *     (3/7) D1^2 psi2 (growth factors are the caller's).
 *
 * Ownership: inputs and outputs are caller-owned; device pointers unless a
 * call says otherwise.  The hierarchy owns its padded working state, allocated
 * through cfg->dev_alloc/dev_free (cudaMalloc/cudaFree when both are NULL) and
 * released by mg_hierarchy_destroy.  Each call is ordered after the work
 * already queued on the caller's stream (given at create time) and the
 * caller's stream is ordered after the call's work; internally the hierarchy
 * runs on its own non-blocking stream so that its cycles can be captured and
 * replayed as CUDA graphs.  The solve calls read one 32-byte convergence record
 * back per V-cycle (so they return with the work finished).
 *
 * Errors: every call returns an mg_status; no exception or abort crosses the
 * ABI.  mg_last_error() gives a message for the last failing call on a handle.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_MAX_LEVELS 16
#define MG_MAX_HISTORY 64

typedef struct mg_hierarchy mg_hierarchy;

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,   /* invalid configuration or argument                        */
  MG_ENOMEM = 2,   /* the allocator returned NULL                              */
  MG_ENOCONV = 3,  /* max_cycles reached above tol; outputs hold the last iterate */
  MG_ECUDA = 4,    /* a CUDA runtime call or kernel launch failed              */
  MG_ETIMEOUT = 5  /* a bounded device-side wait ran out; outputs are invalid    */
} mg_status;

/* MG_FP64: every step in float64.  MG_MIXED: iterative refinement; the
 * residual f - L u, the coarsest-level solve and the update u += e are float64,
 * the correction equation L e = r is solved by float32 V-cycles (smoothing,
 * transfers and coarse-fine ghosts in float32): inner_cycles of them in the first
 * outer iteration; each later one runs just enough cycles to take the float64
 * residual to a quarter of the tolerance at the reduction the previous outer
 * iteration achieved (its first cycle, from a zero correction, counted as 5 times
 * weaker than the others), at most inner_cycles (all inner_cycles when tol = 0);
 * the stopping test is the same float64 leaf residual norm. */
typedef enum { MG_FP64 = 0, MG_MIXED = 1 } mg_precision;

/* MG_FLAG_NO_GRAPHS: launch every kernel on the stream instead of replaying one
 * captured CUDA graph per V-cycle (MG_FP64) or per outer iteration (MG_MIXED). */
#define MG_FLAG_NO_GRAPHS 1
/* Smoother kernel: by default float32 nests of at least 2^23 cells are smoothed
 * by the kernel that stages plane tiles in shared memory with the tensor-memory
 * accelerator, other levels by the kernel that loads every stencil value from
 * global memory; both give bit-identical results.  MG_FLAG_NO_TMA: the second
 * kernel on every level.  MG_FLAG_TMA_ALL: the first kernel on every level. */
#define MG_FLAG_NO_TMA 2
#define MG_FLAG_TMA_ALL 4
/* MG_FLAG_HYBRID: the displacements of mg_lpt_pipeline and mg_batch_lpt_pipeline get
 * the hybrid Poisson solver correction on the finest level (Sec. 3.5.2, see
 * mg_hybrid_correction) with that level's source (delta for psi1, tau for psi2). */
#define MG_FLAG_HYBRID 8
/* MG_FLAG_DEVICE_LOOP: the iteration loop of every solve runs on the device: one
 * CUDA graph per solve whose while node repeats the iteration and whose last
 * kernel applies the stopping rule (and, in MG_MIXED, the inner-cycle plan) of the
 * host loop, so no host round trip separates two iterations.  Same launches and
 * results as the host loop; ignored with MG_FLAG_NO_GRAPHS or while profiling. */
#define MG_FLAG_DEVICE_LOOP 16
/* MG_FLAG_PERSISTENT: in mg_batch_lpt_pipeline, the float32 half of each outer
 * iteration (zero correction, inner V-cycles) of every active MG_MIXED member that sets
 * this flag runs inside ONE persistent kernel launch over a work list of (hierarchy,
 * level operation, block range) items, instead of one launch per level operation per
 * member: each hierarchy's operations form a chain, and a block takes an item only from
 * a chain whose earlier operations have completed (so no block waits on an item it
 * holds); a block that finds nothing to take for 2 s (a defect) stops the launch with
 * MG_ETIMEOUT.  The float64 half (update, ghosts, residual norm) follows on the members'
 * own streams; members without the flag run their per-operation launches concurrently
 * with the persistent launch.  Results are bit-identical to the per-operation launches.
 * Ignored outside a batch. */
#define MG_FLAG_PERSISTENT 32
/* MG_FLAG_PAIR_SMOOTHER: the global-memory float32 smoother updates the cell of colour
 * c of one z-pair per thread on every level.  By default, levels whose rows are a
 * multiple of 4 cells long are smoothed by a kernel that updates the two cells of
 * colour c of one z-quad per thread (one 16-byte load per neighbour row for both);
 * both give bit-identical results. */
#define MG_FLAG_PAIR_SMOOTHER 64

typedef struct {
  int n_levels;                        /* 1 = base only; 1 + number of nests            */
  int base_n[3];                       /* periodic base grid                            */
  double box;                          /* base box length                               */
  int nest_n[MG_MAX_LEVELS - 1][3];    /* nest i (level i+1): size in its own cells     */
  int nest_off[MG_MAX_LEVELS - 1][3];  /* nest i: origin in parent cells                */
  int order;                           /* FD order: 2, 4 or 6                           */
  int precision;                       /* mg_precision                                  */
  int nu1, nu2;                        /* pre/post smoothing sweeps (paper: 2, 2)       */
  int max_cycles;                      /* V-cycle limit per solve (MG_MIXED: outer     */
                                       /* refinement iterations)                        */
  int inner_cycles;                    /* MG_MIXED: float32 V-cycles of the first outer  */
                                       /* iteration and the most of any later one        */
  int flags;                           /* MG_FLAG_* bits; 0 = defaults                  */
  int tile_rows;                       /* smoother block: 32 z-pairs x tile_rows y rows  */
                                       /* (1, 2, 4, 8; 0 = 4)                            */
  double tol;                          /* stop when leaf |r| / leaf |f| <= tol, or when  */
                                       /* |r| <= 64 eps (|f|^2 + V mean^2)^(1/2), the     */
                                       /* rounding level of a constant source             */
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
} mg_config;

typedef struct {
  int cycles;                          /* V-cycles run (MG_MIXED: outer iterations)     */
  double rel_residual;                 /* final leaf |r| / leaf |f|                     */
  double source_mean;                  /* composite mean removed from the source        */
  double history[MG_MAX_HISTORY];      /* rel_residual after each cycle                 */
  int inner_cycles;                    /* MG_MIXED: float32 V-cycles run in total       */
  /* after the last cycle, per leaf level l (0 = base, i = nest i-1): the volume-weighted
   * L2 norm of f - L u over that level's leaf cells divided by the same norm of its f
   * (the norm itself where the level's f is zero); entries >= n_levels are 0.  The
   * largest entry shows where the composite residual sits (Sec. 3.2 stopping rule). */
  double level_rel_residual[MG_MAX_LEVELS];
} mg_info;

/* Fill *cfg with defaults: order 2, FP64, nu1 = nu2 = 2, max_cycles 50,
 * inner_cycles 2, tile_rows 4, tol 1e-10, box 1, no nests, NULL allocator.
 * Host only. */
void mg_config_default(mg_config* cfg);

/* Check the geometry and parameters without touching a GPU.  On failure
 * returns MG_EINVAL and writes a message into msg (if msg != NULL, len > 0). */
mg_status mg_config_validate(const mg_config* cfg, char* msg, size_t len);

/* Device bytes the hierarchy for *cfg allocates (for admission by HBM budget);
 * 0 if the configuration is invalid.  Host only. */
size_t mg_workspace_bytes(const mg_config* cfg);

/* Number of levels (full multigrid coarsenings below the base + base + nests)
 * the V-cycle visits; 0 if invalid.  Host only. */
int mg_total_levels(const mg_config* cfg);

/* Create a hierarchy on the current CUDA device; cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  *out is NULL on failure. */
mg_status mg_hierarchy_create(const mg_config* cfg, void* cuda_stream, mg_hierarchy** out);

/* Free the working state (NULL-safe). */
mg_status mg_hierarchy_destroy(mg_hierarchy* h);

/* Change the caller's stream that later calls are ordered against (a server
 * hands a resident hierarchy to whichever worker stream serves a request). */
mg_status mg_set_stream(mg_hierarchy* h, void* cuda_stream);

/* 1LPT potential (Sec. 3.1.1, 3.2-3.3): solve L phi = delta - <delta>.
 * delta[l], phi[l]: n_levels device pointers, dense float64 per level.
 * info may be NULL. */
mg_status mg_solve_1lpt(mg_hierarchy* h, const double* const delta[], double* const phi[],
                        mg_info* info);

/* 2LPT potential (Sec. 3.1.2): tau(phi1) with FD second derivatives, then
 * L phi2 = tau - <tau>.  phi1 as returned by mg_solve_1lpt. */
mg_status mg_solve_2lpt(mg_hierarchy* h, const double* const phi1[], double* const phi2[],
                        mg_info* info);

/* Displacement psi = -G phi (Sec. 3.1.1, Table 1 gradient) on every level.
 * disp[3*l + a] is component a (x, y, z) of level l, dense float64. */
mg_status mg_displacements(mg_hierarchy* h, const double* const phi[], double* const disp[]);

/* The 2LPT source tau on every level (before mean removal); covered cells hold
 * the average of their children.  Same layout as delta. */
mg_status mg_lpt2_source(mg_hierarchy* h, const double* const phi1[], double* const tau[]);

/* Hybrid Poisson solver correction (Sec. 3.5.2): psi[c] (c = x, y, z; dense device
 * arrays of the finest level) += IFFT[i (k_c / k^2 + g_c / Lt) FFT[f]], the exact
 * k-space gradient of the inverse Laplacian minus its order-n finite-difference
 * counterpart (Table 1 symbols: Lt = -sum_a lam_n(k_a h) / h^2, i g_c = i g_n(k_c h) / h),
 * applied to the finest level's own source f (dense, device), which is zero outside
 * the level: a nest is zero-padded to twice its size; a single periodic level is
 * corrected periodically.  The multiplier is 0 at k = 0 and on the Nyquist plane of
 * axis c.  psi = -G phi, so psi + correction is the exact k-space displacement of
 * the level's own source plus the multigrid long-range part.  Allocates (on first use;
 * kept until mg_hierarchy_destroy) a real and two complex grids of the (padded) level
 * and cuFFT plans.  Errors: MG_EINVAL, MG_ECUDA. */
mg_status mg_hybrid_correction(mg_hierarchy* h, const double* f, double* const psi[3]);

/* Local Lagrangian approximation of the density (Sec. 5.3, eq. for rho(q, t)):
 * rho[l] = rho / rho_bar = 1 / det[delta_ij + dL_i/dq_j] for the displacement
 * L = a1 psi1 + a2 psi2 = -grad(a1 phi1 + a2 phi2) (e.g. a1 = D1, a2 = 3/7 D1^2), i.e.
 * dL_i/dq_j = -Phi_,ij with Phi = a1 phi1 + a2 phi2 and the finite-difference
 * Hessian of the 2LPT source (Phi_,ii: 1D second difference; Phi_,ij: G_i G_j, with
 * edge ghosts on nests).  Covered cells hold the mean of their children; the field
 * is then shifted so that its volume-weighted composite leaf mean is exactly 1
 * (mass conservation).  Where det <= 0 (shell crossing) the approximation does not
 * hold and the result is 1/det as computed.  phi1, rho: device, dense per leaf level;
 * phi2 may be NULL (a2 unused).  Overwrites the hierarchy's float64 state and leaf
 * sources.  Errors: MG_EINVAL (NULL pointers, non-finite a1/a2), MG_ECUDA. */
mg_status mg_lla_density(mg_hierarchy* h, const double* const phi1[], const double* const phi2[],
                         double a1, double a2, double* const rho[]);

/* One whole initial-conditions step: phi1 = solve(delta), phi2 = solve(tau(phi1)),
 * disp1 = -G phi1, disp2 = -G phi2.  host_buffers != 0: every pointer is a host
 * pointer and the call copies inputs in and outputs out on its stream (pinned
 * host memory gives asynchronous copies); otherwise all are device pointers.
 * Any output array pointer may be NULL to skip that output's copy-out. */
mg_status mg_lpt_pipeline(mg_hierarchy* h, int host_buffers, const double* const delta[],
                          double* const phi1[], double* const phi2[], double* const disp1[],
                          double* const disp2[], mg_info* info1, mg_info* info2);

/* 2LPT source tau of one periodic grid, with no device allocation.  The paper
 * has no counterpart; this is for callers that cannot allocate device memory
 * when they need the result (their device memory is held by their own pool,
 * they are given a stream but no allocator, or they must avoid the device
 * synchronisation cudaMalloc/cudaFree can cause).
 *   phi, tau  caller-owned device arrays, dense float64 [n0][n1][n2]
 *   box       length of axis 0 (h = box / n0); order 2, 4 or 6
 *   err       optional message buffer of len bytes
 * Working memory is one static device array of 16 MiB (five ghost-padded grids,
 * about 64^3 cells at order 6); larger grids return MG_EINVAL with a message.
 * The first call on each device looks up the array's address and should be
 * made outside stream capture; the address is kept until the process exits, so
 * the call must not be used on a device after cudaDeviceReset in the same
 * process.  Calls share the array: calls whose work overlaps on the GPU race,
 * so callers serialise them.  Asynchronous on cuda_stream. */
mg_status mg_lpt2_source_periodic_static(const double* phi, double* tau, int n0, int n1,
                                         int n2, double box, int order, void* cuda_stream,
                                         char* err, size_t len);

/* A batch of independent hierarchies solved together (config 4 style: many
 * small, uneven hierarchies).  Each member keeps its own configuration and
 * device state; the V-cycles (MG_FP64) or outer iterations (MG_MIXED) of all
 * members that have not converged are captured into one CUDA graph with one
 * branch per member and replayed with a single launch per iteration, so the
 * members' kernels run concurrently.  Results equal each member's results
 * when solved alone (the same kernels on the same data, no cross-member
 * arithmetic).  Members must not be used elsewhere while the batch runs. */
typedef struct mg_batch mg_batch;

mg_status mg_batch_create(mg_hierarchy* const members[], int count, void* cuda_stream,
                          mg_batch** out);
mg_status mg_batch_destroy(mg_batch* b);

/* mg_lpt_pipeline for every member: delta[i], phi1[i], ... are member i's
 * pointer arrays (as for mg_lpt_pipeline); info1/info2 are arrays of count
 * records (or NULL).  Returns the worst member status; MG_ENOCONV if any member
 * stopped above its tol. */
mg_status mg_batch_lpt_pipeline(mg_batch* b, int host_buffers, const double* const* const delta[],
                                double* const* const phi1[], double* const* const phi2[],
                                double* const* const disp1[], double* const* const disp2[],
                                mg_info* info1, mg_info* info2);

/* Message for the last failing batch call ("" if none; NULL-safe). */
const char* mg_batch_last_error(const mg_batch* b);

/* Grid of the persistent launch (MG_FLAG_PERSISTENT members): blocks_per_sm blocks per
 * SM (1..64, capped at what fits), or 0 (default) for as many as fit, which leaves no
 * room for the concurrent per-operation launches of members without the flag.  Drops
 * the batch's cached graphs.  Errors: MG_EINVAL. */
mg_status mg_batch_set_persistent_blocks(mg_batch* b, int blocks_per_sm);

/* Serving runtime: a request queue in front of resident hierarchies, driven by
 * one native scheduler thread.  A request is mg_lpt_pipeline(host_buffers = 1)
 * for one configuration: the density delta in (preferably pinned) host memory
 * in, phi1, phi2 and both displacement fields out to host memory.
 *  - Admission by HBM budget: a request needs mg_workspace_bytes(cfg) of device
 *    memory for a hierarchy of its configuration; the server keeps the bytes of
 *    its resident hierarchies under the budget, closing idle ones (least
 *    recently used first) to make room.  Each scheduler pass first starts, in
 *    arrival order, the pending requests that find an idle resident hierarchy
 *    of their configuration, then gives the oldest request still waiting a new
 *    hierarchy if it fits (one creation per pass).
 *  - Resident state: hierarchies are cached by configuration (every field of
 *    mg_config), so a repeated configuration reuses its levels and captured
 *    CUDA graphs; overlapping requests of one configuration get one hierarchy
 *    each, budget permitting.
 *  - Overlap without a thread per request: each admitted request runs as a
 *    non-blocking job on its hierarchy's stream; the scheduler polls the event
 *    after the work a job queued last and queues the job's next piece (next
 *    iteration, tau, stores) when it has finished, so up to max_active requests
 *    at different stages share the GPU.
 *  - Results depend only on the request: the same launches as mg_lpt_pipeline
 *    on the same data, so they are bit-identical to a solo call.
 * The device is the one current when mg_server_create is called.  The server
 * owns its hierarchies; the caller owns every buffer of a request, which must
 * stay valid until the request's result has been returned by mg_server_poll. */
typedef struct mg_server mg_server;

typedef struct {
  long long id;        /* the id given to mg_server_submit                         */
  int status;          /* mg_status of the request's pipeline                      */
  mg_info info1, info2;/* convergence records of the 1LPT and 2LPT solves          */
  double t_submit;     /* CLOCK_MONOTONIC seconds: submitted, started on the GPU,   */
  double t_start;      /* results in host memory                                  */
  double t_done;
  char error[160];     /* message of a failed request ("" otherwise)               */
} mg_server_result;

typedef struct {
  unsigned long long resident_bytes;  /* mg_workspace_bytes of resident hierarchies */
  unsigned long long peak_bytes;
  unsigned long long budget_bytes;
  long long created;                  /* hierarchies created                        */
  long long evictions;                /* idle hierarchies closed to make room        */
  long long completed;                /* results handed to the result queue          */
  int pending, active, instances, peak_active;
  /* scheduler thread: CPU seconds (updated every 64 passes and whenever a pass moves
   * nothing), wall seconds of the passes that started, advanced or finished a job,
   * seconds since mg_server_create, and passes made.  Under load a CPU share near 1
   * means the host thread, not the GPU, limits the throughput. */
  double sched_cpu_s, sched_busy_s, uptime_s;
  long long passes;
} mg_server_stats;

/* max_active: requests on the GPU at once (1..256).  Errors: MG_EINVAL, MG_ECUDA. */
mg_status mg_server_create(unsigned long long hbm_budget, int max_active, mg_server** out);

/* Queues one request.  delta: one host pointer per leaf level (base first, dense
 * [nx][ny][nz] float64); phi1, phi2: NULL or one host pointer per leaf level;
 * disp1, disp2: NULL or three per leaf level (x, y, z).  The pointer arrays are
 * copied.  Returns MG_EINVAL (invalid cfg, missing pointers, server closing) or
 * MG_ENOMEM (the hierarchy alone exceeds the budget) without queueing it. */
mg_status mg_server_submit(mg_server* s, long long id, const mg_config* cfg,
                           const double* const delta[], double* const phi1[],
                           double* const phi2[], double* const disp1[], double* const disp2[]);

/* Moves up to max finished requests' results into out (completion order),
 * waiting up to wait_seconds for the first one; returns how many (0 on timeout,
 * -1 for invalid arguments). */
int mg_server_poll(mg_server* s, mg_server_result* out, int max, double wait_seconds);

mg_status mg_server_get_stats(mg_server* s, mg_server_stats* out);

/* At most n resident hierarchies per configuration (n = 0, the default: no cap).  A
 * request whose configuration has n hierarchies, all busy, waits for one of them to
 * be idle instead of getting a new one: creating a hierarchy (device allocation, and
 * the capture of its graphs on first use) stalls the device for every running job,
 * so under load an uncapped server can spend its time making instances.  May be
 * called at any time; takes effect at the scheduler's next pass. */
mg_status mg_server_set_max_instances(mg_server* s, int n);

/* Stops taking requests, fails the ones not yet started (status MG_EINVAL,
 * "server closed"), waits for the running ones, frees every hierarchy.
 * NULL-safe.  Results not yet polled are dropped.  No other mg_server_* call on
 * the same server may run concurrently with it (submit, poll and get_stats may
 * otherwise be called from any threads at once). */
mg_status mg_server_destroy(mg_server* s);

/* Kernel families for launch counting and event timing. */
typedef enum {
  MG_K_SMOOTH = 0,     /* red-black half-sweep                                 */
  MG_K_RESTRICT = 1,   /* residual + restriction, restriction of u             */
  MG_K_FAS = 2,        /* FAS source on covered parent cells                   */
  MG_K_PROLONG = 3,    /* prolongation-correction                              */
  MG_K_GHOST = 4,      /* periodic ghosts, coarse-fine interpolation and flux  */
  MG_K_COARSEST = 5,   /* exact solve on the coarsest level                    */
  MG_K_NORM = 6,       /* residual norms, composite mean, reductions           */
  MG_K_LPT = 7,        /* 2LPT source and gradient                             */
  MG_K_COPY = 8,       /* packing, fills                                       */
  MG_K_FAMILIES = 9
} mg_kernel_family;

typedef struct {
  long long launches[MG_K_FAMILIES];  /* kernel launches since the last reset            */
  long long cells[MG_K_FAMILIES];     /* cells each family processed (smooth: updated)    */
  double event_ms[MG_K_FAMILIES];     /* summed CUDA-event time of timed launches         */
  long long timed[MG_K_FAMILIES];     /* launches that carried events                     */
  long long timed_cells[MG_K_FAMILIES]; /* cells of the launches that carried events      */
} mg_stats;

/* Time launches of the families in mask (bit f = family f) with CUDA event
 * pairs on the hierarchy's stream (0 disables): every launch outside the
 * V-cycle loops, and inside the loops the launches of the first cycle (or
 * outer iteration) of each solve, a sample that visits every level once.
 * mg_stats.timed counts the timed launches. */
mg_status mg_set_profiling(mg_hierarchy* h, unsigned mask);

/* Restrict the event timing of mg_set_profiling to launches that process at least
 * min_cells cells (default 0: every launch), e.g. the largest level's launches of
 * a family.  mg_stats.timed_cells sums the cells of the timed launches. */
mg_status mg_set_profiling_min_cells(mg_hierarchy* h, long long min_cells);

/* Copy the counters out (synchronising the stream to read event times) and,
 * if reset != 0, zero them. */
mg_status mg_get_stats(mg_hierarchy* h, mg_stats* out, int reset);

/* Message for the last failing call on h ("" if none; NULL-safe). */
const char* mg_last_error(const mg_hierarchy* h);

/* Self-test of the device-side wait limit, the failure-detection path of the
 * TMA-staged smoother (no counterpart in the paper).  Runs that kernel once on an
 * internal periodic 16^3 float32 level (order 6) with the byte count expected for
 * its first staged plane raised by 16, so that plane's mbarrier never completes
 * although every copy lands: the block's bounded wait gives up after about 2 s,
 * drains its copies, sets the error flag and returns.  Returns MG_ETIMEOUT when
 * the limit and the error path work, MG_OK if the limit did not trigger (a defect),
 * MG_ENOMEM or MG_ECUDA on a CUDA failure.  Synchronous; allocates and frees its own
 * device memory on the current device; the CUDA context stays usable. */
mg_status mg_selftest_wait_limit(void);

/* Measured issue rate of the FP64 pipe of the current device, the roofline
 * denominator of the float64 stencil kernels (no counterpart in the paper): one
 * warm-up launch, then one timed launch of 8 blocks of 256 threads per SM, each
 * thread running 8 independent chains of `iters` fused multiply-adds (16 <= iters
 * <= 2^22; 4096 takes about 20 ms on a GB300).  *fma_per_s = FP64 FMAs per second.
 * Synchronous on cuda_stream; allocates nothing.  Errors: MG_EINVAL, MG_ECUDA. */
mg_status mg_fp64_fma_rate(int iters, void* cuda_stream, double* fma_per_s);

/* The event-pair floor (no counterpart in the paper): the mean time that a pair of
 * CUDA events reads around one kernel node of a CUDA graph when the kernel does nothing
 * (event record node, a 1-block empty kernel, event record node; `pairs` of them in one
 * graph, 1 <= pairs <= 1024, timed on the graph's second replay).  The profiled kernel
 * families (mg_set_profiling) are timed with the same pairs, so their event-timed
 * durations include this fixed cost; subtracting it bounds a kernel's own duration from
 * below.  *us in microseconds.  Ordered after cuda_stream, synchronous; creates and
 * frees its own graph, stream and events.  Errors: MG_EINVAL, MG_ECUDA. */
mg_status mg_event_pair_floor(int pairs, void* cuda_stream, double* us);

/* Self-test of the persistent batch kernel's bounded dependency wait (no counterpart
 * in the paper): one launch of that kernel on an internal two-item work list whose
 * second item depends on an operation that does not exist, with a 100 ms wait limit.
 * Returns MG_ETIMEOUT when the limit and the error path work, MG_OK if the wait did
 * not give up (a defect), MG_ENOMEM or MG_ECUDA on a CUDA failure.  Synchronous;
 * allocates and frees its own device memory; the CUDA context stays usable. */
mg_status mg_selftest_persist_wait(void);

/* ---- Density generator (Hahn & Abel 2011, Sec. 2.1) ----------------------------
 * Gaussian white noise from a counter-based generator and its periodic
 * convolution with a radial amplitude: delta = IFFT[A(|k|) FFT[noise]], the
 * k-space form of the paper's delta = T * mu on a periodic level. */

/* out[i], i in [0, n): standard normal deviates.  Element i comes from pair index
 * q = i / 2: Philox4x32-10 (Salmon et al. 2011) with counter (q mod 2^32,
 * q div 2^32, 0, 0) and key (seed mod 2^32, seed div 2^32) gives four 32-bit words
 * x0..x3; u1 = ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) / 2^53, u2 likewise from x2, x3;
 * out[2q] = r cos(2 pi u2), out[2q+1] = r sin(2 pi u2), r = sqrt(-2 ln u1).
 * out: device pointer, 16-byte aligned, n doubles.  Asynchronous on cuda_stream.
 * Errors: MG_EINVAL (n < 0, NULL or misaligned out), MG_ECUDA (launch). */
mg_status mg_white_noise(unsigned long long seed, long long n, double* out, void* cuda_stream);

typedef struct mg_field mg_field;  /* opaque: FFT plans and spectrum of one grid size */

/* A generator for periodic n0 x n1 x n2 grids of cubic cells of side h (grid sides
 * 2..4096).  The amplitude A(|k|) is the linear interpolation of amp[0..nt) (host,
 * nt >= 2, finite), sampled at |k| = t dk; A = 0 beyond (nt - 1) dk and at k = 0.
 * For the density of Sec. 2.1 with numpy-style unnormalised transforms, A = sqrt(P(k)
 * / h^3).  Allocates the half spectrum (16 n0 n1 (n2/2+1) bytes) and two cuFFT plans
 * on the current device.  Errors: MG_EINVAL, MG_ENOMEM, MG_ECUDA. */
mg_status mg_field_create(int n0, int n1, int n2, double h, const double* amp, int nt,
                          double dk, mg_field** out);

/* delta = IFFT[A(|k|) FFT[noise]] / (n0 n1 n2 normalisation of the inverse), both
 * dense [x][y][z] doubles on the device (they may be the same buffer).  Asynchronous
 * on cuda_stream; calls on one generator must not overlap (they share its spectrum). */
mg_status mg_field_convolve(mg_field* g, const double* noise, double* delta, void* cuda_stream);

/* delta = the field of the white noise mg_white_noise(seed, n0 n1 n2) (generated in
 * delta itself, then convolved in place). */
mg_status mg_field_generate(mg_field* g, unsigned long long seed, double* delta,
                            void* cuda_stream);

const char* mg_field_last_error(const mg_field* g);  /* "" if none; NULL-safe */

/* Multi-scale density on the nested hierarchy cfg describes (Sec. 2.3), into
 * delta[l] (device, dense per leaf level, base first):
 *  - noise: level l draws mg_white_noise's deviates with counter word 2 = l;
 *  - nests: Hoffman-Ribak constraint (Sec. 2.3.1), the mean of the 8 children of
 *    each parent cell := parent noise / sqrt(8);
 *  - base: periodic field IFFT[A FFT[noise]], A(|k|) = sqrt_p(|k|) / h^{3/2} with
 *    sqrt_p[0..nt) (host) sampled at |k| = t dk as for mg_field_create;
 *  - nest: isolated field of its own noise (zero-padded to twice its size) plus
 *    the parent-level field of all noise outside it (its parent's noise with the
 *    nest region zeroed, convolved like the parent's own, plus what the parent
 *    carried), brought down by conservative tricubic interpolation (tensor cubic
 *    Lagrange through 4 parent cells, then each group of 8 children shifted to
 *    average to the parent value) (Sec. 2.3.3-2.3.4);
 *  - covered cells hold the mean of their 8 children.
 * Allocates its work arrays and cuFFT plans on the current device for the call;
 * synchronous on cuda_stream.  Errors: MG_EINVAL (invalid cfg or table), MG_ENOMEM,
 * MG_ECUDA. */
mg_status mg_density_multiscale(const mg_config* cfg, unsigned long long seed, const double* sqrt_p,
                                int nt, double dk, double* const delta[], void* cuda_stream);
mg_status mg_field_destroy(mg_field* g);             /* NULL-safe */

/* Library version string. */
const char* mg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
