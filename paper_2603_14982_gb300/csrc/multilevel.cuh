// multilevel.cuh -- inter-level transfers and new-block initialisation kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "hierarchy.cuh"
#include "storage.cuh"

namespace hlbm {

constexpr int kMaxLevels = 4;  // most levels a lattice may have

// Read-only view of one level for the transfer kernels.
struct LevelView {
  GridDims d;                 // block grid
  const int32_t* slot;        // [slots] block index or -1
  const int32_t* coords;      // [nb][3]
  const void* mom;            // current buffer
  const void* mom_other;      // the other ping-pong buffer
  int64_t nb;
  const Scales* sc;           // row scales (reduced-precision storage) or null
  BlockHash hash;             // spatial-hash block table, used instead of slot when set
};

struct TransferArgs {
  LevelView fine, coarse;
  void* out;                  // buffer written (fine for down, coarse for up)
  const Scales* out_sc;       // its row scales or null
  const int32_t* nodes;       // (block << 9) | cell of the written level
  int64_t n_nodes;
  int avg;                    // down: 1 = temporal midpoint of coarse mom_other (old) and mom (new)
  int use_other;              // down: 1 = coarse state is mom_other (step 1), 0 = mom
  double k;                   // S^neq factor
  int periodic[3];
  int* status;                // set to 1 if a stencil node is not stored
  const int32_t* stencil;     // down: [8][n_nodes] (coarse block << 9) | cell of each stencil node of
                              // nodes[k], -1 past its stencil, -2 where the coarse node is not stored
  float* undo;                // optional (FP32 storage): the written nodes' previous stored values,
                              // [n_nodes][10] in the order of nodes (the adjoint's undo log)
  double* acc_old;            // down, optional [n_nodes][10]: step 1 stores the FP64 stencil sums of the
                              // old coarse state there; step 2 reuses them instead of re-reading the
                              // old state (it is the same state: the coarse level does not step between)
};

// The stencil table of a downward transfer (a.stencil written through
// `out`): per node of a.nodes its coarse stencil nodes, in the order the
// transfer sums them; sets *a.status to 1 for a coarse node that is not
// stored.  Depends on the hierarchy only.
cudaError_t down_stencil(const TransferArgs& a, int32_t* out, cudaStream_t s);
// DownwardTransfer of Algorithm 1 (Eq. downward_rescale) into I^d nodes of the fine level.
cudaError_t transfer_down(int storage, const TransferArgs& a, cudaStream_t s);
// UpwardTransfer of Algorithm 1 (Eq. upload_S) into I^u nodes of the coarse level.
cudaError_t transfer_up(int storage, const TransferArgs& a, cudaStream_t s);

// Old hierarchy for initialising the moments of a new one at a rebuild.
struct OldHierarchy {
  int L;
  LevelView lv[kMaxLevels];
  double kup[kMaxLevels];    // S^neq factor level l -> l+1
  double kdown[kMaxLevels];  // S^neq factor level l+1 -> l
  int periodic[3];
  int ext[3];                // fine-equivalent extent
};

// Fill the current buffer of new level l: nodes stored before keep their
// moments; the others take the upward rule from the finest old level that
// holds the coincident node, else the downward spatial rule from old coarser
// levels (recursively).  status is set to 1 if a node has no source.
cudaError_t init_new_level(int storage, const OldHierarchy& old, int level, const int32_t* coords, int64_t nb,
                           void* out, const Scales* out_sc, int* status, cudaStream_t s);

// Test hook: the transfers' binary64 -> binary32 narrowing of n device values
// into out, and the conversion instruction's result into hw.
cudaError_t test_narrow(const double* in, float* out, float* hw, int64_t n, cudaStream_t s);

}  // namespace hlbm
