// lattice_state.h -- host-side state behind the opaque hlbm_lattice handle.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hlbm_internal.h"

namespace hlbm {

constexpr int kRescaleEvery = 32;  // steps between scale refreshes of FP16/BF16 storage

// Kernel classes of the per-handle profile (hlbm_set_profiling): stream time
// between CUDA events recorded on the handle's stream around each phase.
enum ProfClass {
  kProfStreamCollide = 0,  // stream-collide of every level (coupled steps included)
  kProfDown,               // downward transfers
  kProfUp,                 // upward transfers
  kProfOpenFaces,          // open-face updates
  kProfRebuild,            // hierarchy rebuilds (whole call)
  kProfDeposit,            // particle deposits
  kProfAdjoint,            // recordings and adjoints (whole calls)
  kProfReduce,             // FP64 reductions
  kProfClasses
};

struct Profile {
  bool on = false;
  struct Span {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Span> pending;       // recorded, not yet read
  std::vector<cudaEvent_t> pool;   // events free for reuse
  double ms[kProfClasses] = {};
  int64_t count[kProfClasses] = {};
};

// One operation of a multi-level coarse step in the order of Algorithm 1,
// with the buffers a recorded or recomputed run gave it.
enum AdjOpKind { kSC, kDown, kUp };
struct AdjOp {
  AdjOpKind kind;
  int l, s;
  void* in = nullptr;       // SC: input state; DOWN: fine state written; UP: coarse state written
  void* out = nullptr;      // SC: output state
  float* pre = nullptr;     // SC: pre-collision moments
  void* c_old = nullptr;    // DOWN: P_{l+1}
  void* c_new = nullptr;    // DOWN: A_{l+1}; UP: the fine state read (A_l)
  float* undo = nullptr;    // DOWN / UP: overwritten values
};

// Reverse-mode tape of the last checkpoint segment (FP32 storage).  The
// recording pass runs that segment with the adjoint's own recomputation, so
// the adjoint starts its reverse walk there without recomputing it; its
// buffers then serve the adjoint as the segment buffers of every other
// segment.  One adjoint consumes the tape (the multi-level reverse walk puts
// the undo logs back into these buffers).
struct AdjTape {
  std::vector<void*> bufs;     // every allocation of the tape
  int n = 0;                   // recorded steps: fine steps (one level), coarse steps (multi-level)
  // one level: seg[i + 1] = state after step i of the segment, pre[i] = its p
  std::vector<void*> seg, pre;
  // multi-level: the segment's operations, the per-level working copy of its
  // start state (the transfers write in place) and the FP64 downward sums
  std::vector<AdjOp> ops;
  std::vector<void*> work;
  std::vector<double*> acc;
};

struct LevelData {
  int64_t nb = 0;                  // stored blocks
  std::vector<int32_t> coords;     // host copy [nb][3] (bx, by, bz), ascending slot id (see host_lists)
  std::vector<uint8_t> flags;      // host copy [nb] leaf/border/new/refine/coarsen bits
  bool host_lists = false;         // coords / flags hold the current lists (copied from the device on
                                   // demand for hierarchies built on the device)
  uint8_t* d_list_flags = nullptr; // [nb] flags of the device-built list
  int32_t* d_nbr = nullptr;        // [nb][27]
  int32_t* d_open = nullptr;       // [nb + 1]: the blocks with an open neighbour, their count last (made
                                   // by the first step with open faces; dropped with the neighbour tables)
  void* d_mom[2] = {nullptr, nullptr};  // ping-pong moment buffers [nb][10][512]
  int cur = 0;                     // buffer holding the current state
  double tau = 0;                  // level relaxation time
  uint8_t* d_bflags = nullptr;     // [nb] step-kernel block flags
  uint32_t* d_bmask = nullptr;     // [nb][512] bounce-back masks
  uint8_t* d_solid = nullptr;      // [nb][512] solid nodes or null
  uint8_t* d_skip = nullptr;       // [nb] 1 = covered by a finer level (left out of reductions) or null
  // hierarchy built on the device (multi-level lattices and rebuilds)
  int32_t* d_coords = nullptr;     // [slots][3] capacity, first nb used
  int32_t* d_slot = nullptr;       // [slots] slot -> block index or -1 (null with a spatial hash)
  unsigned long long* d_hkeys = nullptr;  // spatial-hash block table (block lookup mode 1), else null
  int32_t* d_hvals = nullptr;
  uint32_t hcap = 0;
  uint8_t* d_H = nullptr;          // [slots] block has stored finer children
  uint8_t* d_stored = nullptr;     // [slots] block is stored
  int64_t n_down = 0, n_up = 0;    // interface node counts (I^d, I^u)
  int32_t* d_down = nullptr;       // [n_down] (block << 9) | cell
  int32_t* d_down_t = nullptr;     // [n_down] the same nodes in transfer order (grouped by stencil shape)
  int32_t* d_down_stc = nullptr;   // [8][n_down] their coarse stencil nodes, (block << 9) | cell
  int32_t* d_up = nullptr;         // [n_up]
  double* d_down_acc = nullptr;    // [n_down][10] FP64 stencil sums of the old coarse state (step s = 1,
                                   // reused at s = 2), in transfer order
  // reduced-precision storage: row scales shared by both buffers, a spare
  // Scales for re-encoding, and the amax scratch
  Scales* d_scales = nullptr;      // [2]
  unsigned* d_amax = nullptr;      // [kRows]
  int steps_since_rescale = 0;
};

}  // namespace hlbm

struct hlbm_lattice {
  hlbm_config cfg{};
  cudaStream_t stream = nullptr;
  std::vector<hlbm::LevelData> lv;
  double fu[3] = {0, 0, 0};
  float* d_F = nullptr;    // level-0 force [nb0][3][512] or null
  float* d_eps = nullptr;  // level-0 fluid fraction [nb0][512] or null
  bool have_blocks = false;
  hlbm::Profile prof;
  void* d_stage = nullptr;  // staging for host moment I/O
  size_t stage_bytes = 0;
  double* d_red = nullptr;  // reduction scratch
  size_t red_n = 0;
  bool device_hierarchy = false;  // levels were built by the device rebuild pipeline
  int block_lookup = 0;           // 0: dense per-level slot tables, 1: spatial hash (hlbm_set_block_lookup)
  double kup[8] = {0}, kdown[8] = {0};  // S^neq factors between level l and l+1
  int* d_status = nullptr;    // device status word of the transfer kernels (0 = ok)
  uint8_t* d_prev_occ = nullptr;  // level-0 occupancy the installed hierarchy was built from (particle
                                  // or block-list rebuilds), or null
  unsigned long long* d_count = nullptr;  // scratch counter (particles dropped by a deposit)
  // forward run recorded for the adjoint: states at steps 0, K, 2K, ...
  // (multi-level: one buffer per level and checkpoint, [c * L + l])
  std::vector<void*> ckpt;
  hlbm::AdjTape* tape = nullptr;  // the recorded run's last segment, until an adjoint takes it
  int32_t rec_steps = 0, rec_every = 0;
  int64_t hier_gen = 0;  // bumped whenever the block layout changes
  // live drag of the coupled step (coupling.cu): every drag_every-th level-0
  // step streams, exchanges F = kappa (1 - eps) (vp - u*) and collides
  double drag_kappa = 0, drag_vp[3] = {0, 0, 0};
  int32_t drag_every = 0;
  int64_t l0_steps = 0;  // level-0 steps since hlbm_set_drag
  // open faces (boundary.cu), order x-, x+, y-, y+, z-, z+: HLBM_FACE_CLOSED,
  // HLBM_FACE_OUTFLOW or HLBM_FACE_INLET; inlet profile u0 ln(1 + beta (h - h0))
  // along axis inlet_axis (fine-node units)
  int32_t face_type[6] = {0, 0, 0, 0, 0, 0};
  double inlet_u0 = 0, inlet_beta = 0, inlet_h0 = 0;
  int32_t inlet_axis = 1;
  unsigned open_mask() const {
    unsigned m = 0;
    for (int f = 0; f < 6; ++f)
      if (face_type[f] != 0) m |= 1u << f;
    return m;
  }
  int64_t rec_gen = -1;  // hier_gen of the recorded run
  // hlbm_set_blocks: block lists of the levels staged since the last
  // installed explicit hierarchy ([level] -> coordinates; staged[level] set)
  std::vector<std::vector<int32_t>> staged_blocks;
  std::vector<uint8_t> staged;
  std::string err;

  void block_dims(int level, int dims[3]) const {
    const int s = 8 << level;
    dims[0] = cfg.nx / s;
    dims[1] = cfg.ny / s;
    dims[2] = cfg.nz / s;
  }
};

namespace hlbm {
// Records one span of class `cls` on h->stream while profiling is on.
class ProfScope {
 public:
  ProfScope(hlbm_lattice* h, int cls);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  hlbm_lattice* h_;
  int cls_;
  cudaEvent_t a_ = nullptr;
};
// Reads every finished span into the totals (synchronises the stream).
int profile_collect(hlbm_lattice* h);
}  // namespace hlbm

namespace hlbm {

// Records an error message on h (or the global one when h is NULL) and returns code.
int fail(hlbm_lattice* h, int code, const char* fmt, ...);

// True when the device allocation about to be made is the one that
// hlbm_inject_alloc_failure asked to fail (consumes one count otherwise).
bool alloc_failure_injected();

// Multi-level engine (ml_host.cu).
// H_given: per level, the has-children set on the dense slot grid (level 0
// all zero); when set, the occupancy inputs are ignored and the hierarchy
// follows from these sets.
int ml_rebuild(hlbm_lattice* h, const float* pos, int64_t n_pos, int pos_on_device, const int32_t* blocks,
               int64_t n_blocks, int64_t counts_out[3],
               const std::vector<std::vector<uint8_t>>* H_given = nullptr);
// Stage the explicit block list of one level (hlbm_set_blocks); installs the
// hierarchy once every level is staged.
int ml_set_blocks(hlbm_lattice* h, int level, const int32_t* coords_xyz, int64_t n);
int ml_advance_coarse(hlbm_lattice* h, int64_t n_coarse);
int ml_check_status(hlbm_lattice* h);
// Reverse mode of the multi-level advance, FP32 storage (adjoint_ml.cu):
// record n_steps fine steps with a checkpoint of every level each ckpt_every
// fine steps (both multiples of 2^(L-1)), then the adjoint from dL/dM of the
// final state (levels concatenated) to dL/dF of the level-0 force.
int ml_forward_record(hlbm_lattice* h, int32_t n_steps, int32_t ckpt_every);
// The coupled level-0 step (coupling.cu): is the next level-0 step an
// exchange step, and the step itself (a: level-0 arguments with in / out).
bool exchange_due(const hlbm_lattice* h);
int coupled_step(hlbm_lattice* h, const StepArgs& a);
// Open faces (boundary.cu): after a step of `level` from `in` to `out`, write
// the open-face nodes of `out` from the state `in` (no-op without open faces).
int open_faces_step(hlbm_lattice* h, int level, const void* in, void* out);
int ml_adjoint(hlbm_lattice* h, const float* dL_dM, float* dL_dF);

struct LatticeOps {
  static int set_device(hlbm_lattice* h);
  static int alloc(hlbm_lattice* h, void** p, size_t bytes);
  static void release(hlbm_lattice* h, void*& p);
  static void free_level(hlbm_lattice* h, LevelData& L);
  static void release_tape(hlbm_lattice* h);
  // Allocate the scale state of a reduced-precision level (scales for amax 0).
  static int init_scales(hlbm_lattice* h, LevelData& L);
  // Re-derive a reduced-precision level's scales every kRescaleEvery steps.
  static int maybe_rescale(hlbm_lattice* h, LevelData& L, bool force);
  // (Re)compute d_bflags / d_bmask of a level from its neighbour table and solids.
  static int bounce(hlbm_lattice* h, LevelData& L);
  // Make L.coords / L.flags current (one device-to-host copy after a rebuild).
  static int host_lists(hlbm_lattice* h, LevelData& L);
  static int open_lists(hlbm_lattice* h);
  static void build_nbr(const hlbm_lattice* h, int level, const std::vector<int32_t>& coords,
                        const std::vector<int32_t>& slot_to_idx, std::vector<int32_t>& nbr);
};

}  // namespace hlbm
