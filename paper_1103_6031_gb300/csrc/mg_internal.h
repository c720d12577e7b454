// Internal declarations shared by the CUDA translation units of the library.
//
// Device layout of one level: the interior n0 x n1 x n2 cells plus a ghost
// shell of width g = order/2 on every side, row-major [x][y][z] with z fastest.
// Along z the interior starts at element za = 4 (>= g) and rows are padded to
// a pitch Zp that is a multiple of 8 elements, so every interior row starts on
// a 32-byte boundary and even z indices allow 16-byte vector access for
// float64 (and 16-byte access for groups of 4 at z = 0 mod 4 for float32).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg.h"

namespace mgk {

struct Grid {
  int n0, n1, n2;  // interior extent
  int g;           // ghost width
  int za;          // z index of the first interior element within a row
  int Y;           // padded extent along y (n1 + 2g)
  int Zp;          // row pitch in elements
  int X;           // padded extent along x (n0 + 2g)
};

__host__ __device__ inline long long gidx(const Grid& G, int i, int j, int k) {
  return ((long long)(i + G.g) * G.Y + (j + G.g)) * G.Zp + (k + G.za);
}

inline long long grid_elems(const Grid& G) { return (long long)G.X * G.Y * G.Zp; }

// Ghost cells of a periodic level's shell (the periodic ghost fill's thread count).
__host__ __device__ inline long long ghost_shell_count(const Grid& G) {
  const long long g = G.g;
  const long long X = G.n0 + 2 * g, Y = G.n1 + 2 * g;
  return X * Y * 2 * g + X * 2 * g * G.n2 + 2 * g * (long long)G.n1 * G.n2;
}

Grid make_grid(int n0, int n1, int n2, int g);

struct Int3 {
  int x, y, z;
};

// Interpolation weights for the coarse-fine ghost zones, computed on the host
// from their Lagrange definition (see mg_weights.cpp).
struct CfWeights {
  double tang[2][7];   // [fine parity][parent offset -half..half]
  double ncoarse[3][3];  // [ghost layer m][coarse node q]
  double nfine[3][4];    // [ghost layer m][fine node q]
  double flux[6];        // face-flux weights on cells face-half .. face+half-1
  double ghost_coef[2];  // sum of flux weights on the ghost side: [low face, high face]
};

void compute_cf_weights(int order, CfWeights* w);

// Geometry of the 6 faces of a nest for the face kernels.
struct FaceSet {
  int nt[6][2];         // tangential extents (fine cells) of face f: axes b, c
  long long base[7];    // prefix sums of half * nt0 * nt1 (intermediate values per face)
  long long ebase[7];   // prefix sums of (nt0/2) * (nt1/2) (parent face elements per face)
};

void make_faceset(const Grid& F, int half, FaceSet* fs);

// ---- kernels: smoothing and inter-level transfer (mg_smooth.cu) ----
// quad: float32 levels whose rows are a multiple of 4 long take the z-quad kernel
// (bit-identical to the z-pair kernel taken otherwise).
template <typename T>
cudaError_t launch_smooth_half(int order, const Grid& G, const T* uin, T* uout, const T* f,
                               double a_f, int colour, int periodic, int rows, bool quad,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_residual_restrict(int order, const Grid& F, const T* u, const T* f,
                                     double invh2, const Grid& P, T* pu, T* pfas, T* ubar,
                                     Int3 off, Int3 cn, int parent_periodic, cudaStream_t s);
template <typename T>
cudaError_t launch_fas_source(int order, const Grid& P, const T* pu, T* pfas, double invH2,
                              Int3 off, Int3 cn, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong(const Grid& F, T* u, const Grid& P, const T* pu, const T* ubar,
                           Int3 off, Int3 cn, int periodic, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict_u(const Grid& F, const T* u, const Grid& P, T* pu, Int3 off,
                              Int3 cn, cudaStream_t s);

// ---- TMA-staged smoother (mg_smooth_tma.cu) ----
// Same update and result as launch_smooth_half; the input buffer u is read through
// tin, the source f through tf (both made by make_plane_tmap, with halo = true for
// u and false for f).  *err is or-ed with 1 when a block's wait for a staged plane
// ran out.  extra_tx > 0 (wait-limit self-test only) raises the byte count expected
// for the first staged plane so that its wait runs out.
template <typename T>
cudaError_t launch_smooth_half_tma(int order, const Grid& G, const CUtensorMap* tin,
                                   const CUtensorMap* tf, T* uout, double a_f, int colour,
                                   int periodic, unsigned* err, cudaStream_t s,
                                   unsigned extra_tx = 0);
// Tensor map of one padded level buffer (elem_bytes 4 or 8) for the plane boxes of
// the TMA smoother: with halo, 72 x (8 + order) elements of z x y; without, 64 x 8.
cudaError_t make_plane_tmap(const Grid& G, const void* base, int elem_bytes, int order,
                            bool halo, CUtensorMap* tm);
bool smooth_tma_usable(const Grid& G);
// Opt the TMA smoother kernels in to their shared-memory size on the current device.
cudaError_t prepare_smooth_tma();

// ---- kernels: ghost zones (mg_ghost.cu) ----
template <typename T>
cudaError_t launch_ghost_periodic(const Grid& G, T* u, cudaStream_t s);
template <typename T>
cudaError_t launch_cf_tangential(int order, const Grid& F, const Grid& P, const T* pu, Int3 off,
                                 const FaceSet& fs, const CfWeights& w, double invH, T* inter,
                                 T* fc_unc, cudaStream_t s);
template <typename T>
cudaError_t launch_cf_flux(int order, const Grid& F, T* u, const FaceSet& fs, const CfWeights& w,
                           const T* inter, const T* fc_unc, double h, double invh, double invH,
                           int flux_fix, cudaStream_t s);
template <typename T>
cudaError_t launch_cf_edges(int order, const Grid& F, T* u, const Grid& P, const T* pu, Int3 off,
                            const CfWeights& w, cudaStream_t s);

// ---- kernels: coarsest solve, norms, packing, 2LPT, gradient (mg_misc.cu) ----
cudaError_t launch_coarsest(const Grid& G, const double* f, double* u, const double* kern,
                            cudaStream_t s);
// float32 source and result, float64 arithmetic (mixed precision keeps the coarsest
// solve in float64)
cudaError_t launch_coarsest(const Grid& G, const float* f, float* u, const double* kern,
                            cudaStream_t s);
// partial sums over uncovered interior cells of level G: [2*b] = sum r^2, [2*b+1] = sum f^2
// (times vol), r = f - L u; blocks = number of partial slots written.
// With r32 != nullptr the residual of every interior cell is also written to r32
// (float32, same layout) as the source of the mixed-precision correction equation.
cudaError_t launch_norm_partial(int order, const Grid& G, const double* u, const double* f,
                                double invh2, double vol, Int3 clo, Int3 chi, double* partial,
                                int blocks, float* r32, cudaStream_t s);
cudaError_t launch_add_correction(const Grid& G, double* u, const float* e, int periodic,
                                  cudaStream_t s);
// p[0..n) -= sum[0] * scale, with sum on the device
cudaError_t launch_sub_mean(double* p, long long n, const double* sum, double scale,
                            cudaStream_t s);
cudaError_t launch_sum_partial(const Grid& G, const double* f, double vol, Int3 clo, Int3 chi,
                               double* partial, int blocks, cudaStream_t s);
cudaError_t launch_reduce_partials(const double* partial, int count, int width, double* out,
                                   cudaStream_t s);
// Slots [off[l], off[l] + cnt[l]) of the partial-sum array belong to leaf level l.
struct LevelRanges {
  int n;
  int off[MG_MAX_LEVELS];
  int cnt[MG_MAX_LEVELS];
};
// out[0..1] = the sums of all `count` pairs (the same order as launch_reduce_partials);
// out_levels[2 l .. 2 l + 1] = the sums of leaf level l's pairs.
cudaError_t launch_reduce_levels(const double* partial, int count, const LevelRanges& R,
                                 double* out, double* out_levels, cudaStream_t s);
cudaError_t launch_pack(const Grid& G, const double* src, double* dst, double shift,
                        cudaStream_t s);
// dense dst = padded interior of src + add
cudaError_t launch_unpack(const Grid& G, const double* src, double* dst, cudaStream_t s,
                          double add = 0.0);
cudaError_t launch_shift_copy(const Grid& G, double* f, double* f2, const double* mean_num,
                              double inv_volume, cudaStream_t s);
cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t s);
// tau from phi (ghosts, including edges, filled); work holds 3 * grid_elems(G)
// float64 for the first derivatives.
cudaError_t launch_lpt2_source(int order, const Grid& G, const double* phi, double invh2,
                               double* tau, double* work, cudaStream_t s);
// 1/det[I - H] - 1 on the interior (H: finite-difference Hessian of phi, ghosts and
// edges filled); work holds 3 * grid_elems(G) float64.
cudaError_t launch_lla(int order, const Grid& G, const double* phi, double invh2, double* out,
                       double* work, cudaStream_t s);
// out = a1 x1 + a2 x2 over n dense elements (x2 may be NULL)
cudaError_t launch_axpby(long long n, double a1, const double* x1, double a2, const double* x2,
                         double* out, cudaStream_t s);
cudaError_t launch_gradient(int order, const Grid& G, const double* phi, double invh, double* dx,
                            double* dy, double* dz, cudaStream_t s);

int norm_blocks(const Grid& G);

// ---- hybrid Poisson solver correction (mg_hybrid.cu) ----
struct HybridFFT;
// Plans and buffers for an n0 x n1 x n2 level of spacing h (pad: zero-padded to 2x).
cudaError_t hybrid_create(HybridFFT** out, int n0, int n1, int n2, double h, int order,
                          bool pad);
void hybrid_destroy(HybridFFT* hy);
// psi[c] (dense, device) += the correction of source f (dense, device), c = 0, 1, 2.
cudaError_t hybrid_apply(HybridFFT* hy, const double* f, double* const psi[3], cudaStream_t s);
// device bytes of hybrid_create for that level (buffers and an estimate of cuFFT's work area)
size_t hybrid_bytes(int n0, int n1, int n2, bool pad);

// ---- non-blocking pipelines (mg_api.cu), driven by the server (mg_serve.cu) ----
// mg_lpt_pipeline(host_buffers = 1) on h as a job that never waits for the GPU:
// job_start queues the loads and the first iteration; job_poll advances the job
// when the work it queued last has finished: it returns 0 (still waiting), 1 (the
// next piece is queued) or 2 (finished: every result is in the caller's host
// buffers and nothing is in flight).
// The pointer arrays are copied; the buffers must stay valid until then.  The
// hierarchy serves one job at a time.  job_start returns MG_EINVAL (and makes no
// job) for missing pointers; a job that fails later finishes with that status.
struct PipelineJob;
mg_status job_start(mg_hierarchy* h, const double* const delta[], double* const phi1[],
                    double* const phi2[], double* const disp1[], double* const disp2[],
                    PipelineJob** out);
int job_poll(PipelineJob* j);
mg_status job_result(const PipelineJob* j, mg_info* info1, mg_info* info2);
const char* job_error(const PipelineJob* j);
void job_destroy(PipelineJob* j);

}  // namespace mgk
