// lattice_state.h -- host-side state behind the opaque hlbm_lattice handle.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hlbm_internal.h"

namespace hlbm {

struct LevelData {
  int64_t nb = 0;                  // stored blocks
  std::vector<int32_t> coords;     // host copy [nb][3] (bx, by, bz), ascending slot id
  std::vector<uint8_t> flags;      // host copy [nb] leaf/border/new/refine/coarsen bits
  int32_t* d_nbr = nullptr;        // [nb][27]
  void* d_mom[2] = {nullptr, nullptr};  // ping-pong moment buffers [nb][10][512]
  int cur = 0;                     // buffer holding the current state
  double tau = 0;                  // level relaxation time
  uint8_t* d_bflags = nullptr;     // [nb] step-kernel block flags or null
  uint8_t* d_solid = nullptr;      // [nb][512] solid nodes or null
  uint8_t* d_skip = nullptr;       // [nb] 1 = covered by a finer level (left out of reductions) or null
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
  void* d_stage = nullptr;  // staging for host moment I/O
  size_t stage_bytes = 0;
  double* d_red = nullptr;  // reduction scratch
  size_t red_n = 0;
  std::string err;

  void block_dims(int level, int dims[3]) const {
    const int s = 8 << level;
    dims[0] = cfg.nx / s;
    dims[1] = cfg.ny / s;
    dims[2] = cfg.nz / s;
  }
};

namespace hlbm {

struct LatticeOps {
  static int set_device(hlbm_lattice* h);
  static int alloc(hlbm_lattice* h, void** p, size_t bytes);
  static void release(void*& p);
  static void free_level(LevelData& L);
  static void build_nbr(const hlbm_lattice* h, int level, const std::vector<int32_t>& coords,
                        const std::vector<int32_t>& slot_to_idx, std::vector<int32_t>& nbr);
};

}  // namespace hlbm
