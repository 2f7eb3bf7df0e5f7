// hlbm_internal.h -- internal interfaces between the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/homelbm.h"
#include "storage.cuh"

namespace hlbm {

// Neighbour-table sentinels: a stored block index is >= 0.
constexpr int32_t kMissing = -1;  // inside the domain but not stored at this level
constexpr int32_t kWall = -2;     // beyond a non-periodic face of the domain
constexpr int32_t kOpen = -3;     // beyond an open face (convective outflow or inlet)

// A neighbour block whose nodes the step cannot pull from: the nodes that
// touch it keep their moments in the stream-collide step (interface nodes,
// filled by a transfer; open-face nodes, filled by the boundary update).
__host__ __device__ constexpr bool is_copy_nbr(int32_t v) { return v == kMissing || v == kOpen; }

// Per-block flag bits of the step kernel.
constexpr uint8_t kBlockSolidNear = 1;  // the block or one of its 26 neighbours holds a solid node
constexpr uint8_t kBlockBounce = 2;     // some node of the block pulls from a wall or a solid node

// Arguments of one stream-collide launch over the stored blocks of a level.
struct StepArgs {
  const void* in;           // storage [nb][10][512]
  void* out;                // storage [nb][10][512]
  const int32_t* nbr;       // [nb][27] neighbour block per direction (dx+1)+3(dy+1)+9(dz+1)
  const float* F;           // [nb][3][512] force, or null (uniform fu)
  const float* eps;         // [nb][512] fluid fraction, or null (1)
  const uint8_t* solid;     // [nb][512] solid node mask, or null
  const uint8_t* bflags;    // [nb] block flags, or null
  const uint32_t* bmask;    // [nb][512] bounce-back masks (bit k: pull source x - c_k is wall/solid)
  const Scales* scales_in;  // reduced-precision row scales of `in` (device), else null
  const Scales* scales_out; // row scales of `out` (device), else null
  double fu[3];             // uniform force when F is null
  double tau;               // level relaxation time
  double om;                // 1 / tau
  double kxyz;              // third-order xyz weight (27 or 13.5)
  int64_t nb;               // number of blocks processed by the launch
  int64_t blk0;             // first block index of the launch (0: all)
  const float* blk_om;      // [nb_total] per-block 1/tau (batches of domains), or null (om)
  const int32_t* blk_dom;   // [nb_total] per-block domain index into scales_in/out, or null
  unsigned* work;           // non-null: persistent launch of `grid` CTAs over a ticket counter
                            // (two zeroed unsigned in device memory, left zeroed); FP32/FP16/BF16 only
  int grid;
  // float copies of fu, tau, om, kxyz for the FP32-math kernel (set by its launcher:
  // FP64 conversions run on the slow FP64 pipe, so the kernel takes floats)
  float fuf[3], tauf, omf, kxyzf;
  float* pre_out;           // [nb][10][512] float32 natural order: pre-collision moments (recording launch)
};

// FP64 storage: one node per thread (stream_collide.cu).  Other storages: the
// packed-FP32 node-pair kernel (stream_collide_f2.cu).
cudaError_t launch_stream_collide(int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_stream_collide_f2(int storage, const StepArgs& a, cudaStream_t s);
// FP32 storage: the step that also writes the pre-collision moments p to
// a.pre_out (forward steps recomputed by the adjoint).
cudaError_t launch_stream_collide_record(const StepArgs& a, cudaStream_t s);
// FP32 / FP16 / BF16 storage: the streaming-only step S of a coupled step,
// writing the pre-collision moments to a.pre_out (float32 natural order) and
// no output state (coupling.cu collides).
cudaError_t launch_stream_only(int storage, const StepArgs& a, cudaStream_t s);
// Resident CTAs per SM of the persistent node-pair kernel.
cudaError_t persistent_ctas_per_sm(int storage, int* per_sm);
// One reverse step of the single-level stream-collide, FP64 storage (adjoint.cu): lam = dL/dM
// of the step's output, lam_out = dL/dM of its input (a.in), dF += dL/dF.
// lamp is scratch [nb][10][512]; all lambda arrays are natural node order.
cudaError_t adjoint_step(int storage, const StepArgs& a, const float* lam, float* lamp, double* dF, float* lam_out,
                         cudaStream_t s);
cudaError_t adjoint_dF_to_float(const double* dF, float* out, int64_t n, cudaStream_t s);
// FP32 storage, reverse step from recorded pre-collision moments: adjoint_collide
// (elementwise: lamp = (dC/dp)^T lam, dF += (dC/dF)^T lam unless dF is null;
// solid and interface nodes get lamp = 0) then adjoint_push (lam_out = dL/dM
// of the step's input a.in; solid nodes copy lam, interface nodes add it to
// what streams back; lam_add, if set, is added at every node and, with
// clear_add, left zero behind).
cudaError_t adjoint_collide(const StepArgs& a, const float* pre, const float* lam, float* lamp, double* dF,
                            cudaStream_t s, float* dFs = nullptr);
cudaError_t adjoint_push(const StepArgs& a, const float* lam, const float* lamp, float* lam_out, cudaStream_t s,
                         float* lam_add = nullptr, bool clear_add = false);
// adjoint_push of a step fused with adjoint_collide of the step before it
// (recorded p = pre_prev): writes that step's lamp to lamp_out, adds to dF.
// The step's own lam_out is stored only at the pass-through (solid and
// interface) nodes, into raw_out if it is set; lam, lam_add and clear_add as
// for adjoint_push (raw_out may equal lam).
cudaError_t adjoint_push_collide(const StepArgs& a, const float* lamp, const float* pre_prev, float* lamp_out,
                                 double* dF, cudaStream_t s, const float* lam = nullptr, float* raw_out = nullptr,
                                 float* lam_add = nullptr, bool clear_add = false, float* dFs = nullptr);
// dFs (FP32, [nb][3][512]), where a call takes it, receives the force terms
// instead of dF: the sum over one checkpoint segment.  adjoint_dF_flush adds
// it to the FP64 dF and zeroes it.
cudaError_t adjoint_dF_flush(double* dF, float* dFs, int64_t n, cudaStream_t s);

// Per-node bounce masks and the kBlockBounce flag from a neighbour table and
// an optional solid mask (bflags must hold kBlockSolidNear where solids are near).
cudaError_t compute_bounce_masks(const int32_t* nbr, const uint8_t* solid, uint8_t* bflags, uint32_t* bmask,
                                 int64_t nb, cudaStream_t s);

}  // namespace hlbm
