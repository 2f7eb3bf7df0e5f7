// hierarchy.cuh -- device-side block-hierarchy maintenance (Sec. 5.4, Sec. 6.1, Sec. 6.3).
//
// All sets live on dense per-level slot grids (uint8 per block slot, slot id
// bz*(nby*nbx) + by*nbx + bx).  The rules are the declarative ones:
//   O_0      level-0 blocks holding a particle (Phi = 0 there)
//   H_1      = dilate(parent(O_0)),  H_l = dilate(parent(H_{l-1}))
//   I_l      = {b in H_l : every in-domain 26-neighbour in H_l}
//   stored_l = children(H_{l+1}) \ I_l  (l < L-1),  all \ I_{L-1} (top)
//   border   = stored and (in H_l or parent stored), else leaf
// Stored blocks are compacted in ascending slot order with warp ballots and a
// block-level scan, which makes the lists unique and order-stable.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hlbm {

struct GridDims {
  int nx, ny, nz;  // blocks per axis
  __host__ __device__ int64_t slots() const { return int64_t(nx) * ny * nz; }
};

constexpr uint8_t kFlagLeaf = 1, kFlagBorder = 2, kFlagNew = 4, kFlagRefine = 8, kFlagCoarsen = 16;

// Spatial-hash variant of a level's block table (Sec. 6.1: the active tiles
// of each level are found by position through a spatial hash): open
// addressing with linear probing over a power-of-two table of 64-bit keys
// (bz << 42 | by << 21 | bx; all ones = empty), at most half full.  The slot
// of a key is the SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014)
// of the key, masked.
constexpr unsigned long long kEmptyKey = ~0ull;
struct BlockHash {
  const unsigned long long* keys = nullptr;  // null: the level uses its dense slot table
  const int32_t* vals = nullptr;
  uint32_t mask = 0;  // capacity - 1
};

__host__ __device__ inline unsigned long long block_key(int bx, int by, int bz) {
  return (static_cast<unsigned long long>(bz) << 42) | (static_cast<unsigned long long>(by) << 21) |
         static_cast<unsigned long long>(bx);
}

__host__ __device__ inline uint32_t hash_slot(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return static_cast<uint32_t>(z ^ (z >> 31));
}

// Block index at block coordinates (bx, by, bz) inside the grid, or -1.
__device__ inline int64_t hash_find(const BlockHash& h, int bx, int by, int bz) {
  const unsigned long long key = block_key(bx, by, bz);
  uint32_t s = hash_slot(key) & h.mask;
  for (uint32_t i = 0; i <= h.mask; ++i) {
    const unsigned long long k = h.keys[s];
    if (k == key) return h.vals[s];
    if (k == kEmptyKey) return -1;
    s = (s + 1u) & h.mask;
  }
  return -1;
}

// Dense slot table (all slots -1, then slot of block i = i) from a compacted level.
cudaError_t slot_table(const int32_t* coords, int64_t nb, GridDims d, int32_t* slot_to_idx, cudaStream_t s);
// Capacity of the hash table of a level with nb blocks: a power of two >= 2 nb.
uint32_t hash_capacity(int64_t nb);
// Fill keys (all set to kEmptyKey first) and vals from a compacted level.
cudaError_t build_block_hash(const int32_t* coords, int64_t nb, unsigned long long* keys, int32_t* vals,
                             uint32_t capacity, cudaStream_t s);

// Occupancy of level-0 blocks from particle positions (fine-cell units, x y z
// float32); non-finite positions are counted in *bad and ignored.
cudaError_t occupancy_from_particles(const float* pos, int64_t n, GridDims d0, uint8_t* occ, int* bad, cudaStream_t s);
// Occupancy from an explicit list of level-0 block coordinates (device, [n][3]).
cudaError_t occupancy_from_blocks(const int32_t* coords, int64_t n, GridDims d0, uint8_t* occ, int* bad,
                                  cudaStream_t s);
// H = dilate(parent(src)) on the coarser grid `d` (src lives on the 2x finer grid).
cudaError_t dilate_parent(const uint8_t* src, GridDims dsrc, uint8_t* H, GridDims d, const int periodic[3],
                          cudaStream_t s);
// internal and stored sets of one level; Hup = H of level l+1 (null at the top).
cudaError_t internal_stored(const uint8_t* H, const uint8_t* Hup, GridDims d, GridDims dup, const int periodic[3],
                            bool has_H, uint8_t* I, uint8_t* stored, cudaStream_t s);
// Per-slot flags (0 for slots that are not stored).
cudaError_t slot_flags(const uint8_t* stored, const uint8_t* H, const uint8_t* stored_up, GridDims d, GridDims dup,
                       const uint8_t* old_stored, const uint8_t* old_H, bool has_old, uint8_t* flags,
                       cudaStream_t s);
// Stable compaction of stored slots: slot_to_idx[slot] = index or -1, coords[idx] = (bx,by,bz),
// list_flags[idx] = flags[slot], skip[idx] = H[slot] (covered by finer).  *count written to
// count_dev (device int64).  scratch: >= ceil(slots/1024)+1 int64.
cudaError_t compact_slots(const uint8_t* stored, const uint8_t* flags, const uint8_t* H, GridDims d,
                          int32_t* slot_to_idx, int32_t* coords, uint8_t* list_flags, uint8_t* skip,
                          int64_t* scratch, int64_t* count_dev, cudaStream_t s);
// Neighbour table [nb][27] from a compacted level (open_mask: bit 2 axis + side
// marks an open face; neighbours beyond it are kOpen instead of kWall).
// slot_to_idx null: neighbours found through hash instead.
cudaError_t neighbour_table(const int32_t* coords, int64_t nb, const int32_t* slot_to_idx, GridDims d,
                            const int periodic[3], unsigned open_mask, int32_t* nbr, cudaStream_t s,
                            BlockHash hash = BlockHash{});
// Interface node lists of one level: nodes with a 26-neighbour in a block that
// is not stored; those inside H blocks (skip != 0) go to `up` (I^u), the others
// to `down` (I^d).  Entries are (block << 9) | cell, ascending.
// interface_count writes per-block offsets to scratch (>= 2*nb int64) and the
// totals (down, up) to counts_dev; interface_scatter then fills the lists.
cudaError_t interface_count(const int32_t* nbr, const uint8_t* skip, int64_t nb, int64_t* scratch,
                            int64_t* counts_dev, cudaStream_t s);
cudaError_t interface_scatter(const int32_t* nbr, const uint8_t* skip, int64_t nb, const int64_t* scratch,
                              int32_t* down, int32_t* up, cudaStream_t s);

// Transfer order of a downward interface list: the same n entries grouped by
// the parity class of the node (x, y, z odd or even: the shape of its
// downward stencil), stable within a class.  scratch holds
// transfer_order_scratch(n) int64.
cudaError_t transfer_order(const int32_t* nodes, int64_t n, int64_t* scratch, int32_t* out, cudaStream_t s);
int64_t transfer_order_scratch(int64_t n);

// Adds to *count the positions where a and b (n bytes each) differ.
cudaError_t count_diff(const uint8_t* a, const uint8_t* b, int64_t n, unsigned long long* count, cudaStream_t s);

// Keeps only the leaf / border bits of n list flags (an unchanged hierarchy:
// nothing is new, refined or coarsened).
cudaError_t clear_change_flags(uint8_t* flags, int64_t n, cudaStream_t s);

// Adds to counts_dev[0..3] the slots newly in H (refined), newly out of H
// (coarsened), stored before but not now (deleted) and stored now but not
// before (added) on one level's grid.
cudaError_t count_changes(const uint8_t* H_new, const uint8_t* H_old, const uint8_t* stored_new,
                          const uint8_t* stored_old, int64_t slots, unsigned long long* counts_dev, cudaStream_t s);

}  // namespace hlbm
