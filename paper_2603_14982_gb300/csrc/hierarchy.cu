// hierarchy.cu -- block-hierarchy maintenance on the device (Sec. 5.4, Sec. 6.1, Sec. 6.3).
#include "hierarchy.cuh"
#include "hlbm_internal.h"

namespace hlbm {
namespace {

constexpr int kScanCta = 1024;  // slots per compaction CTA

__device__ __forceinline__ int64_t slot_of(const GridDims& d, int x, int y, int z) {
  return (int64_t(z) * d.ny + y) * d.nx + x;
}

// Wrap (periodic) or reject (wall) a coordinate along one axis.
__device__ __forceinline__ bool wrap(int& v, int n, int periodic) {
  if (v >= 0 && v < n) return true;
  if (!periodic) return false;
  v = (v % n + n) % n;
  return true;
}

__global__ void k_occ_particles(const float* __restrict__ pos, int64_t n, GridDims d0, uint8_t* occ, int* bad) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
  if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) {
    atomicAdd(bad, 1);
    return;
  }
  // floor(p / 8): the division by a power of two is exact
  int bx = int(floorf(px * 0.125f)), by = int(floorf(py * 0.125f)), bz = int(floorf(pz * 0.125f));
  bx = min(max(bx, 0), d0.nx - 1);
  by = min(max(by, 0), d0.ny - 1);
  bz = min(max(bz, 0), d0.nz - 1);
  occ[slot_of(d0, bx, by, bz)] = 1;  // benign race: every writer stores 1
}

__global__ void k_occ_blocks(const int32_t* __restrict__ c, int64_t n, GridDims d0, uint8_t* occ, int* bad) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int bx = c[3 * i], by = c[3 * i + 1], bz = c[3 * i + 2];
  if (bx < 0 || by < 0 || bz < 0 || bx >= d0.nx || by >= d0.ny || bz >= d0.nz) {
    atomicAdd(bad, 1);
    return;
  }
  occ[slot_of(d0, bx, by, bz)] = 1;
}

// H[q] = 1 iff some q' in the 3x3x3 neighbourhood of q (wrapped / clipped) has a
// child set in src (src on the 2x finer grid).
__global__ void k_dilate_parent(const uint8_t* __restrict__ src, GridDims ds, uint8_t* __restrict__ H, GridDims d,
                                int px, int py, int pz) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= d.slots()) return;
  const int x = int(q % d.nx), y = int((q / d.nx) % d.ny), z = int(q / (int64_t(d.nx) * d.ny));
  // all loads independent (no early exit): the two x-children of a child row
  // are one aligned 16-bit word (the finer grid is 2 d.nx wide)
  unsigned hit = 0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        int a = x + dx, b = y + dy, c = z + dz;
        if (!wrap(a, d.nx, px) || !wrap(b, d.ny, py) || !wrap(c, d.nz, pz)) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int cy = 2 * b + (k & 1), cz = 2 * c + (k >> 1);
          hit |= __ldg(reinterpret_cast<const uint16_t*>(src + slot_of(ds, 2 * a, cy, cz)));
        }
      }
  H[q] = hit ? 1 : 0;
}

__global__ void k_internal_stored(const uint8_t* __restrict__ H, const uint8_t* __restrict__ Hup, GridDims d,
                                  GridDims du, int px, int py, int pz, int has_H, uint8_t* __restrict__ I,
                                  uint8_t* __restrict__ stored) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= d.slots()) return;
  const int x = int(q % d.nx), y = int((q / d.nx) % d.ny), z = int(q / (int64_t(d.nx) * d.ny));
  uint8_t in = 0;
  if (has_H && H[q]) {
    in = 1;
    for (int dz = -1; dz <= 1 && in; ++dz)
      for (int dy = -1; dy <= 1 && in; ++dy)
        for (int dx = -1; dx <= 1 && in; ++dx) {
          int a = x + dx, b = y + dy, c = z + dz;
          if (!wrap(a, d.nx, px) || !wrap(b, d.ny, py) || !wrap(c, d.nz, pz)) continue;  // beyond a wall
          in = H[slot_of(d, a, b, c)];
        }
  }
  I[q] = in;
  const uint8_t cover = Hup == nullptr ? 1 : Hup[slot_of(du, x >> 1, y >> 1, z >> 1)];
  stored[q] = (cover && !in) ? 1 : 0;
}

__global__ void k_slot_flags(const uint8_t* __restrict__ stored, const uint8_t* __restrict__ H,
                             const uint8_t* __restrict__ stored_up, GridDims d, GridDims du,
                             const uint8_t* __restrict__ old_stored, const uint8_t* __restrict__ old_H, int has_old,
                             uint8_t* __restrict__ flags) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= d.slots()) return;
  if (!stored[q]) {
    flags[q] = 0;
    return;
  }
  const int x = int(q % d.nx), y = int((q / d.nx) % d.ny), z = int(q / (int64_t(d.nx) * d.ny));
  const uint8_t h = H ? H[q] : 0;
  bool border = h != 0;
  if (stored_up) border = border || stored_up[slot_of(du, x >> 1, y >> 1, z >> 1)] != 0;
  uint8_t f = border ? kFlagBorder : kFlagLeaf;
  if (has_old) {
    const uint8_t oh = old_H ? old_H[q] : 0;
    if (!old_stored[q]) f |= kFlagNew;
    if (h && !oh) f |= kFlagRefine;
    if (!h && oh) f |= kFlagCoarsen;
  }
  flags[q] = f;
}

// Stable compaction, pass 1: per-CTA count of set slots (warp ballots + popc).
__global__ void __launch_bounds__(kScanCta) k_compact_count(const uint8_t* __restrict__ stored, int64_t n,
                                                            int64_t* __restrict__ cta_count) {
  __shared__ int warp_cnt[kScanCta / 32];
  const int64_t i = int64_t(blockIdx.x) * kScanCta + threadIdx.x;
  const bool v = i < n && stored[i];
  const unsigned b = __ballot_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kScanCta / 32; ++w) s += warp_cnt[w];
    cta_count[blockIdx.x] = s;
  }
}

// Exclusive scan of the CTA counts (one CTA, sequential over chunks).
__global__ void k_compact_scan(int64_t* __restrict__ cta_count, int64_t n_cta, int64_t* __restrict__ total) {
  if (threadIdx.x != 0) return;
  int64_t run = 0;
  for (int64_t c = 0; c < n_cta; ++c) {
    const int64_t v = cta_count[c];
    cta_count[c] = run;
    run += v;
  }
  *total = run;
}

// Pass 2: scatter in slot order.
__global__ void __launch_bounds__(kScanCta) k_compact_scatter(const uint8_t* __restrict__ stored,
                                                              const uint8_t* __restrict__ flags,
                                                              const uint8_t* __restrict__ H, GridDims d,
                                                              const int64_t* __restrict__ cta_off,
                                                              int32_t* __restrict__ slot_to_idx,
                                                              int32_t* __restrict__ coords,
                                                              uint8_t* __restrict__ list_flags,
                                                              uint8_t* __restrict__ skip) {
  __shared__ int warp_off[kScanCta / 32];
  const int64_t n = d.slots();
  const int64_t i = int64_t(blockIdx.x) * kScanCta + threadIdx.x;
  const bool v = i < n && stored[i];
  const unsigned b = __ballot_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31;
  if (lane == 0) warp_off[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kScanCta / 32; ++w) {
      const int c = warp_off[w];
      warp_off[w] = s;
      s += c;
    }
  }
  __syncthreads();
  if (i >= n) return;
  if (!v) {
    slot_to_idx[i] = -1;
    return;
  }
  const int64_t idx = cta_off[blockIdx.x] + warp_off[threadIdx.x >> 5] + __popc(b & ((1u << lane) - 1u));
  slot_to_idx[i] = int32_t(idx);
  coords[3 * idx + 0] = int32_t(i % d.nx);
  coords[3 * idx + 1] = int32_t((i / d.nx) % d.ny);
  coords[3 * idx + 2] = int32_t(i / (int64_t(d.nx) * d.ny));
  list_flags[idx] = flags[i];
  skip[idx] = H ? H[i] : 0;
}

// Bit 2 a + side of open_mask: the low (side 0) or high (side 1) face of axis
// a is open.  A neighbour beyond a non-periodic face is kOpen if any face it
// lies beyond is open, else kWall.
__device__ __forceinline__ unsigned beyond_faces(int v, int n, int axis) {
  return v < 0 ? 1u << (2 * axis) : (v >= n ? 2u << (2 * axis) : 0u);
}

__global__ void k_nbr(const int32_t* __restrict__ coords, int64_t nb, const int32_t* __restrict__ slot_to_idx,
                      GridDims d, int px, int py, int pz, unsigned open_mask, int32_t* __restrict__ nbr,
                      BlockHash hash) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= nb * 27) return;
  const int64_t b = i / 27;
  const int dir = int(i % 27);
  int x = coords[3 * b] + dir % 3 - 1, y = coords[3 * b + 1] + (dir / 3) % 3 - 1, z = coords[3 * b + 2] + dir / 9 - 1;
  const unsigned faces = beyond_faces(x, d.nx, 0) | beyond_faces(y, d.ny, 1) | beyond_faces(z, d.nz, 2);
  if (!wrap(x, d.nx, px) || !wrap(y, d.ny, py) || !wrap(z, d.nz, pz)) {
    nbr[i] = (faces & open_mask) != 0u ? kOpen : kWall;
    return;
  }
  // -1 (kMissing) when not stored
  nbr[i] = slot_to_idx != nullptr ? slot_to_idx[slot_of(d, x, y, z)] : int32_t(hash_find(hash, x, y, z));
}

__global__ void k_hash_insert(const int32_t* __restrict__ coords, int64_t nb, unsigned long long* keys,
                              int32_t* vals, uint32_t mask) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const unsigned long long key = block_key(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
  uint32_t s = hash_slot(key) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {  // the table is at most half full
    const unsigned long long prev = atomicCAS(keys + s, kEmptyKey, key);
    if (prev == kEmptyKey || prev == key) {
      vals[s] = int32_t(i);
      return;
    }
    s = (s + 1u) & mask;
  }
}

// Node classification per block (one CTA of 512 threads): a node is an
// interface node iff its 26-neighbourhood touches a missing neighbour block.
__device__ __forceinline__ bool node_missing(int cell, unsigned miss) {
  const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
  const unsigned mx = 2u | (x == 0 ? 1u : 0u) | (x == 7 ? 4u : 0u);
  const unsigned my = 2u | (y == 0 ? 1u : 0u) | (y == 7 ? 4u : 0u);
  const unsigned mz = 2u | (z == 0 ? 1u : 0u) | (z == 7 ? 4u : 0u);
  unsigned touched = 0;
  for (int iz = 0; iz < 3; ++iz)
    for (int iy = 0; iy < 3; ++iy)
      if (((mz >> iz) & 1u) && ((my >> iy) & 1u)) touched |= mx << (3 * iy + 9 * iz);
  return (touched & miss) != 0u;
}

__device__ __forceinline__ unsigned block_missing_mask(const int32_t* nbr, int64_t b) {
  unsigned m = 0;
  for (int d = 0; d < 27; ++d)
    if (nbr[b * 27 + d] == kMissing) m |= 1u << d;
  return m;
}

// counts[2*b] = #down nodes of block b, counts[2*b+1] = #up nodes.
__global__ void __launch_bounds__(512) k_iface_count(const int32_t* __restrict__ nbr, const uint8_t* __restrict__ skip,
                                                     int64_t nb, int64_t* __restrict__ counts) {
  __shared__ unsigned s_miss;
  __shared__ int s_cnt[16];
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) s_miss = block_missing_mask(nbr, b);
  __syncthreads();
  const bool m = s_miss != 0u && node_missing(threadIdx.x, s_miss);
  const unsigned bal = __ballot_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < 16; ++w) s += s_cnt[w];
    const bool up = skip[b] != 0;
    counts[2 * b] = up ? 0 : s;
    counts[2 * b + 1] = up ? s : 0;
  }
}

// Exclusive scan of the (down, up) counts of nb blocks in place, totals to
// totals[0..1]: one CTA, each thread scans a contiguous run of blocks.
__global__ void __launch_bounds__(1024) k_iface_scan(int64_t* __restrict__ counts, int64_t nb,
                                                     int64_t* __restrict__ totals) {
  __shared__ int64_t s_d[32], s_u[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = min(nb, int64_t(t) * per), b1 = min(nb, b0 + per);
  int64_t sd = 0, su = 0;
  for (int64_t b = b0; b < b1; ++b) {
    sd += counts[2 * b];
    su += counts[2 * b + 1];
  }
  int64_t id = sd, iu = su;  // inclusive warp scan
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t vd = __shfl_up_sync(0xffffffffu, id, o), vu = __shfl_up_sync(0xffffffffu, iu, o);
    if (lane >= o) {
      id += vd;
      iu += vu;
    }
  }
  if (lane == 31) {
    s_d[w] = id;
    s_u[w] = iu;
  }
  __syncthreads();
  if (w == 0) {
    int64_t xd = lane < nw ? s_d[lane] : 0, xu = lane < nw ? s_u[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t vd = __shfl_up_sync(0xffffffffu, xd, o), vu = __shfl_up_sync(0xffffffffu, xu, o);
      if (lane >= o) {
        xd += vd;
        xu += vu;
      }
    }
    s_d[lane] = xd;  // inclusive over warps
    s_u[lane] = xu;
  }
  __syncthreads();
  int64_t rd = (w > 0 ? s_d[w - 1] : 0) + id - sd, ru = (w > 0 ? s_u[w - 1] : 0) + iu - su;
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t cd = counts[2 * b], cu = counts[2 * b + 1];
    counts[2 * b] = rd;
    counts[2 * b + 1] = ru;
    rd += cd;
    ru += cu;
  }
  if (t == 0) {
    totals[0] = s_d[nw - 1];
    totals[1] = s_u[nw - 1];
  }
}

__global__ void __launch_bounds__(512) k_iface_scatter(const int32_t* __restrict__ nbr,
                                                       const uint8_t* __restrict__ skip, int64_t nb,
                                                       const int64_t* __restrict__ offs, int32_t* __restrict__ down,
                                                       int32_t* __restrict__ up) {
  __shared__ unsigned s_miss;
  __shared__ int s_off[16];
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) s_miss = block_missing_mask(nbr, b);
  __syncthreads();
  const bool m = s_miss != 0u && node_missing(threadIdx.x, s_miss);
  const unsigned bal = __ballot_sync(0xffffffffu, m);
  const int lane = threadIdx.x & 31;
  if (lane == 0) s_off[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < 16; ++w) {
      const int c = s_off[w];
      s_off[w] = s;
      s += c;
    }
  }
  __syncthreads();
  if (!m) return;
  const bool isup = skip[b] != 0;
  const int64_t base = offs[2 * b + (isup ? 1 : 0)];
  const int64_t k = base + s_off[threadIdx.x >> 5] + __popc(bal & ((1u << lane) - 1u));
  const int32_t v = int32_t((b << 9) | threadIdx.x);
  if (isup)
    up[k] = v;
  else
    down[k] = v;
}

__global__ void k_count_changes(const uint8_t* __restrict__ hn, const uint8_t* __restrict__ ho,
                                const uint8_t* __restrict__ sn, const uint8_t* __restrict__ so, int64_t n,
                                unsigned long long* out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool in = i < n;
  const unsigned r = __ballot_sync(0xffffffffu, in && hn[i] && !ho[i]);
  const unsigned c = __ballot_sync(0xffffffffu, in && !hn[i] && ho[i]);
  const unsigned d = __ballot_sync(0xffffffffu, in && so[i] && !sn[i]);
  const unsigned a = __ballot_sync(0xffffffffu, in && sn[i] && !so[i]);
  if ((threadIdx.x & 31) == 0) {
    if (r) atomicAdd(out + 0, (unsigned long long)__popc(r));
    if (c) atomicAdd(out + 1, (unsigned long long)__popc(c));
    if (d) atomicAdd(out + 2, (unsigned long long)__popc(d));
    if (a) atomicAdd(out + 3, (unsigned long long)__popc(a));
  }
}

__global__ void k_count_diff(const uint8_t* __restrict__ a, const uint8_t* __restrict__ b, int64_t n,
                             unsigned long long* count) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const unsigned m = __ballot_sync(0xffffffffu, i < n && a[i] != b[i]);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, (unsigned long long)__popc(m));
}

__global__ void k_clear_change_flags(uint8_t* __restrict__ f, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) f[i] = uint8_t(f[i] & (kFlagLeaf | kFlagBorder));
}

inline unsigned grid_for(int64_t n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace

cudaError_t count_diff(const uint8_t* a, const uint8_t* b, int64_t n, unsigned long long* count, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_count_diff<<<grid_for(n, 256), 256, 0, s>>>(a, b, n, count);
  return cudaGetLastError();
}

cudaError_t clear_change_flags(uint8_t* flags, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_clear_change_flags<<<grid_for(n, 256), 256, 0, s>>>(flags, n);
  return cudaGetLastError();
}

cudaError_t occupancy_from_particles(const float* pos, int64_t n, GridDims d0, uint8_t* occ, int* bad,
                                     cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(occ, 0, size_t(d0.slots()), s);
  if (e != cudaSuccess || n == 0) return e;
  k_occ_particles<<<grid_for(n, 256), 256, 0, s>>>(pos, n, d0, occ, bad);
  return cudaGetLastError();
}

cudaError_t occupancy_from_blocks(const int32_t* coords, int64_t n, GridDims d0, uint8_t* occ, int* bad,
                                  cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(occ, 0, size_t(d0.slots()), s);
  if (e != cudaSuccess || n == 0) return e;
  k_occ_blocks<<<grid_for(n, 256), 256, 0, s>>>(coords, n, d0, occ, bad);
  return cudaGetLastError();
}

cudaError_t dilate_parent(const uint8_t* src, GridDims dsrc, uint8_t* H, GridDims d, const int periodic[3],
                          cudaStream_t s) {
  k_dilate_parent<<<grid_for(d.slots(), 256), 256, 0, s>>>(src, dsrc, H, d, periodic[0], periodic[1], periodic[2]);
  return cudaGetLastError();
}

cudaError_t internal_stored(const uint8_t* H, const uint8_t* Hup, GridDims d, GridDims dup, const int periodic[3],
                            bool has_H, uint8_t* I, uint8_t* stored, cudaStream_t s) {
  k_internal_stored<<<grid_for(d.slots(), 256), 256, 0, s>>>(H, Hup, d, dup, periodic[0], periodic[1], periodic[2],
                                                             has_H ? 1 : 0, I, stored);
  return cudaGetLastError();
}

cudaError_t slot_flags(const uint8_t* stored, const uint8_t* H, const uint8_t* stored_up, GridDims d, GridDims dup,
                       const uint8_t* old_stored, const uint8_t* old_H, bool has_old, uint8_t* flags,
                       cudaStream_t s) {
  k_slot_flags<<<grid_for(d.slots(), 256), 256, 0, s>>>(stored, H, stored_up, d, dup, old_stored, old_H,
                                                        has_old ? 1 : 0, flags);
  return cudaGetLastError();
}

cudaError_t compact_slots(const uint8_t* stored, const uint8_t* flags, const uint8_t* H, GridDims d,
                          int32_t* slot_to_idx, int32_t* coords, uint8_t* list_flags, uint8_t* skip,
                          int64_t* scratch, int64_t* count_dev, cudaStream_t s) {
  const int64_t n = d.slots();
  const int64_t n_cta = (n + kScanCta - 1) / kScanCta;
  k_compact_count<<<unsigned(n_cta), kScanCta, 0, s>>>(stored, n, scratch);
  k_compact_scan<<<1, 32, 0, s>>>(scratch, n_cta, count_dev);
  k_compact_scatter<<<unsigned(n_cta), kScanCta, 0, s>>>(stored, flags, H, d, scratch, slot_to_idx, coords,
                                                         list_flags, skip);
  return cudaGetLastError();
}

cudaError_t neighbour_table(const int32_t* coords, int64_t nb, const int32_t* slot_to_idx, GridDims d,
                            const int periodic[3], unsigned open_mask, int32_t* nbr, cudaStream_t s,
                            BlockHash hash) {
  if (nb == 0) return cudaSuccess;
  if (slot_to_idx == nullptr && hash.keys == nullptr) return cudaErrorInvalidValue;
  k_nbr<<<grid_for(nb * 27, 256), 256, 0, s>>>(coords, nb, slot_to_idx, d, periodic[0], periodic[1], periodic[2],
                                                open_mask, nbr, hash);
  return cudaGetLastError();
}

namespace {
__global__ void k_slot_scatter(const int32_t* __restrict__ coords, int64_t nb, GridDims d, int32_t* slot_to_idx) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < nb) slot_to_idx[slot_of(d, coords[3 * i], coords[3 * i + 1], coords[3 * i + 2])] = int32_t(i);
}
}  // namespace

cudaError_t slot_table(const int32_t* coords, int64_t nb, GridDims d, int32_t* slot_to_idx, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(slot_to_idx, 0xff, size_t(d.slots()) * sizeof(int32_t), s);
  if (e != cudaSuccess || nb == 0) return e;
  k_slot_scatter<<<grid_for(nb, 256), 256, 0, s>>>(coords, nb, d, slot_to_idx);
  return cudaGetLastError();
}

uint32_t hash_capacity(int64_t nb) {
  uint32_t c = 64;
  while (int64_t(c) < 2 * nb && c < (1u << 31)) c <<= 1;
  return c;
}

cudaError_t build_block_hash(const int32_t* coords, int64_t nb, unsigned long long* keys, int32_t* vals,
                             uint32_t capacity, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(keys, 0xff, size_t(capacity) * sizeof(unsigned long long), s);
  if (e != cudaSuccess || nb == 0) return e;
  k_hash_insert<<<grid_for(nb, 256), 256, 0, s>>>(coords, nb, keys, vals, capacity - 1u);
  return cudaGetLastError();
}

cudaError_t interface_count(const int32_t* nbr, const uint8_t* skip, int64_t nb, int64_t* scratch,
                            int64_t* counts_dev, cudaStream_t s) {
  if (nb == 0) return cudaMemsetAsync(counts_dev, 0, 2 * sizeof(int64_t), s);
  k_iface_count<<<unsigned(nb), 512, 0, s>>>(nbr, skip, nb, scratch);
  k_iface_scan<<<1, 1024, 0, s>>>(scratch, nb, counts_dev);
  return cudaGetLastError();
}

cudaError_t interface_scatter(const int32_t* nbr, const uint8_t* skip, int64_t nb, const int64_t* scratch,
                              int32_t* down, int32_t* up, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  k_iface_scatter<<<unsigned(nb), 512, 0, s>>>(nbr, skip, nb, scratch, down, up);
  return cudaGetLastError();
}

namespace {

// Transfer order of an interface list ------------------------------------------
// The downward transfer's stencil has 1, 2, 4 or 8 coarse nodes depending on
// the parity of the fine node's coordinates (even: one node on that axis, odd:
// two).  Listed in block order, one warp mixes all eight parity classes and
// runs as long as its widest stencil; ordered by class, a warp's lanes share
// one stencil shape.  The order is stable within a class (block order), so
// that neighbouring lanes still read neighbouring coarse nodes.

constexpr int kOrdThreads = 256, kOrdPer = 8, kOrdTile = kOrdThreads * kOrdPer;

__device__ __forceinline__ int parity_class(int32_t v) {
  const int c = v & 511;  // cell = x + 8 y + 64 z: the parities are bits 0, 3 and 6
  return (c & 1) | ((c >> 2) & 2) | ((c >> 4) & 4);
}

// counts[c * n_tile + t] = entries of class c in tile t (kOrdTile entries).
__global__ void __launch_bounds__(kOrdThreads) k_order_count(const int32_t* __restrict__ nodes, int64_t n,
                                                             int64_t n_tile, int64_t* __restrict__ counts) {
  __shared__ int s_cnt[8];
  if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kOrdTile;
#pragma unroll
  for (int i = 0; i < kOrdPer; ++i) {
    const int64_t e = base + i * kOrdThreads + threadIdx.x;
    if (e < n) atomicAdd(&s_cnt[parity_class(nodes[e])], 1);
  }
  __syncthreads();
  if (threadIdx.x < 8) counts[threadIdx.x * n_tile + blockIdx.x] = s_cnt[threadIdx.x];
}

// Exclusive scan of m values in place, total to *total: one CTA, each thread
// a contiguous run.
__global__ void __launch_bounds__(1024) k_scan_runs(int64_t* __restrict__ v, int64_t m, int64_t* __restrict__ total) {
  __shared__ int64_t s_w[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  const int64_t per = (m + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = min(m, int64_t(t) * per), b1 = min(m, b0 + per);
  int64_t own = 0;
  for (int64_t i = b0; i < b1; ++i) own += v[i];
  int64_t inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t x = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += x;
  }
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t x = lane < nw ? s_w[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_w[lane] = x;
  }
  __syncthreads();
  int64_t run = (w > 0 ? s_w[w - 1] : 0) + inc - own;
  for (int64_t i = b0; i < b1; ++i) {
    const int64_t c = v[i];
    v[i] = run;
    run += c;
  }
  if (t == 0) *total = s_w[nw - 1];
}

// Scatter in class-major, then list order: entry order within a tile is
// (i, warp, lane), the order of the count pass.
__global__ void __launch_bounds__(kOrdThreads) k_order_scatter(const int32_t* __restrict__ nodes, int64_t n,
                                                               int64_t n_tile, const int64_t* __restrict__ offs,
                                                               int32_t* __restrict__ out) {
  constexpr int kW = kOrdThreads / 32;
  __shared__ int s_cnt[kW][8];
  __shared__ int64_t s_off[kW][8];
  __shared__ int64_t s_run[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < 8) s_run[threadIdx.x] = offs[threadIdx.x * n_tile + blockIdx.x];
  const int64_t base = int64_t(blockIdx.x) * kOrdTile;
  for (int i = 0; i < kOrdPer; ++i) {
    const int64_t e = base + i * kOrdThreads + threadIdx.x;
    const bool valid = e < n;
    const int32_t v = valid ? nodes[e] : 0;
    const int c = valid ? parity_class(v) : -1;
    int rank = 0;
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const unsigned bal = __ballot_sync(0xffffffffu, c == cc);
      if (c == cc) rank = __popc(bal & ((1u << lane) - 1u));
      if (lane == 0) s_cnt[w][cc] = __popc(bal);
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      int64_t run = s_run[threadIdx.x];
      for (int ww = 0; ww < kW; ++ww) {
        s_off[ww][threadIdx.x] = run;
        run += s_cnt[ww][threadIdx.x];
      }
      s_run[threadIdx.x] = run;
    }
    __syncthreads();
    if (valid) out[s_off[w][c] + rank] = v;
    __syncthreads();
  }
}

}  // namespace

cudaError_t transfer_order(const int32_t* nodes, int64_t n, int64_t* scratch, int32_t* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t n_tile = (n + kOrdTile - 1) / kOrdTile;
  k_order_count<<<unsigned(n_tile), kOrdThreads, 0, s>>>(nodes, n, n_tile, scratch);
  k_scan_runs<<<1, 1024, 0, s>>>(scratch, 8 * n_tile, scratch + 8 * n_tile);
  k_order_scatter<<<unsigned(n_tile), kOrdThreads, 0, s>>>(nodes, n, n_tile, scratch, out);
  return cudaGetLastError();
}

int64_t transfer_order_scratch(int64_t n) { return 8 * ((n + kOrdTile - 1) / kOrdTile) + 1; }

cudaError_t count_changes(const uint8_t* H_new, const uint8_t* H_old, const uint8_t* stored_new,
                          const uint8_t* stored_old, int64_t slots, unsigned long long* counts_dev, cudaStream_t s) {
  if (slots == 0) return cudaSuccess;
  k_count_changes<<<grid_for(slots, 256), 256, 0, s>>>(H_new, H_old, stored_new, stored_old, slots, counts_dev);
  return cudaGetLastError();
}

}  // namespace hlbm
