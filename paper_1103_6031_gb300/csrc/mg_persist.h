// Work list of the persistent batch kernel (mg_persist.cu): the float32 V-cycles of
// many hierarchies as one launch.  Each hierarchy's level operations (the launches its
// own V-cycles would make: smoother half-sweeps, coarse-fine ghosts, residual and
// restriction, FAS source, coarsest solve, tangential interpolation, prolongation,
// zero fills) form a chain; an operation's blocks are cut into work items, and items
// of any hierarchy run as soon as that hierarchy's earlier operations have completed,
// so every hierarchy advances at once while each one's chain keeps its order.
#pragma once

#include "mg_internal.h"

namespace mgk {

enum POpKind : int {
  P_ZERO = 0,        // out0[0, n) = 0
  P_SMOOTH,          // colour half-sweep: in0 = uin, out0 = uout, in1 = f_fas
  P_CF_FLUX,         // coarse-fine ghosts of a nest: out0 = u, in0 = inter, in1 = fc_unc
  P_GHOST_PERIODIC,  // periodic ghost shell of out0
  P_RESTRICT,        // residual + restriction: in0 = u, in1 = f, out0 = parent u,
                     // out1 = parent f_fas, out2 = ubar
  P_FAS,             // FAS source: in0 = parent u, out0 = parent f_fas
  P_COARSEST,        // exact coarsest solve: in0 = f_fas, out0 = u, kern
  P_TANG,            // tangential interpolation: in0 = parent u, out0 = inter, out1 = fc_unc
  P_PROLONG,         // prolongation-correction: out0 = u, in0 = parent u, in1 = ubar
  P_KINDS
};

// Blocks of a P_ZERO operation cover kZeroPerBlock floats each.
constexpr long long kZeroPerBlock = 4096;
// Threads of every work item (every operation runs as 128-thread blocks).
constexpr int kPersistThreads = 128;

struct POp {
  int kind, order, member, seq;  // seq: position in the member's chain
  int nblk;                      // blocks of the operation
  int per_tile;                  // blocks per work item
  int ntiles;                    // work items
  int gx, gy;                    // 3D operations: blocks along x, y (z = nblk / (gx gy))
  long long tile0;               // first work item of this operation in the launch
  Grid F, P;                     // the level written (F) and its parent (P) where used
  Int3 off, cn;
  int colour, periodic;
  float s[5];                    // float scalars, as the stream launcher rounds them
  const float* in0;
  const float* in1;
  float* out0;
  float* out1;
  float* out2;
  const double* kern;
  long long n;                   // P_ZERO: elements
  FaceSet fs;
};

// Device state of one launch: reset to zero before every launch.
struct PState {
  unsigned finished;  // chains (hierarchies) whose every operation has completed
  unsigned err;       // 1: a bounded wait ran out (or the self-test's limit)
};

// The persistent launch.  ops: every member's chain, member-major (member m's
// operations are ops[mop0[m] .. mop0[m] + mops[m]), in chain order, with seq = position
// in the chain and tile0 = the chain-local number of the operation's first item);
// members: entries of mop0/mops (a member not in this launch has mops = 0); active:
// members with work; wts[member]: float weights; per member done[] (completed
// operations), per operation taken[] (item tickets handed out) and count[] (items
// completed), all zero at launch.  wait_ns bounds the time a block may find nothing to take; running
// out sets st->err and every block stops.
cudaError_t launch_persist(const POp* ops, const int* mop0, const int* mops, int members,
                           int active, const void* wts, PState* st, int* done, int* taken,
                           int* count, unsigned long long wait_ns, int grid, cudaStream_t s);
// After a persistent launch: or 1 into *flags[i] (each non-null) when st->err is set,
// so that every member's convergence read reports the timeout.
cudaError_t launch_persist_flags(const PState* st, unsigned* const* flags, int n, cudaStream_t s);
// Blocks of the persistent kernel that fit on the device at once.
cudaError_t persist_grid(int* grid);
// Bytes of one member's float weights (the CfW<float> of mg_vbody.cuh).
size_t persist_weight_bytes();
// Fills the float weights of a member (dst: persist_weight_bytes() bytes, host).
void persist_weights(const CfWeights& w, void* dst);

}  // namespace mgk
