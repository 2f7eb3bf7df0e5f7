// f2_common.cuh -- building blocks of the node-pair kernels (FP32 math on
// packed pairs of nodes (z, z + 4) of an 8^3 block, 256 threads per block):
// the padded destination-indexed shared population buffer and its pushes
// (own pairs, halo pairs reflected onto the lower face of each axis,
// bounce-back), the gather, and the assignment of halo pairs to threads.  Used by the forward
// stream-collide kernel and by the reverse-step kernels of the adjoint.
#pragma once
#include <utility>

#include "hlbm_internal.h"
#include "lbm_math.cuh"
#include "storage.cuh"
#include "v2.cuh"

namespace hlbm {
namespace f2 {

constexpr int kThreads = 256;
constexpr int kHaloPairs = 244;

// Destination-indexed shared population buffer: one padded plane per
// direction j (the rest plane is not used, so that the reflection of a face
// shifts every canonical direction by the same number of planes); node
// (x, y, z) of the block at pidx(x, y, z) of plane j, which starts at
// j kPlane.  Rows y = -1, 8 and slabs z = -1, 8 are padding that pushes
// leaving the block through a y or z face write and nothing reads; pushes
// leaving through an x face are predicated off.  Padding is shared where it
// can be: row y = 8 of slab z overlaps row y = -1 of slab z + 1 (slab stride
// kPZ = 73 < 10 rows of 8), and slab z = 8 of plane j overlaps slab z = -1 of
// plane j + 1 (plane stride 9 slabs), so padding writes may land on each
// other but never on a node's slot.  This keeps the buffer at 71 KB, which
// leaves room beside two CTAs' buffers for a 60 KB L1 (the staging of the
// halo loads).  Every access of a node is at a compile-time offset from one
// base address, the 32 lanes of a warp touch 32 consecutive words for the
// own pushes and the gather, and kPZ is odd so that the x-face halo stores
// (lanes along y and z) meet at most two to a bank.
constexpr int kPY = 8, kPZ = 73, kPlane = 9 * kPZ;
__host__ __device__ constexpr int pidx(int x, int y, int z) { return x + kPY * (y + 1) + kPZ * (z + 1); }
constexpr size_t kBufBytes = size_t(26 * kPlane + pidx(7, 8, 8) + 1) * sizeof(float);
// plane offset of the mirror image of a canonical direction (component +1 on
// the face axis) along axis ax: its index is lower by 2, 6 or 18
__host__ __device__ constexpr int mirror_shift(int ax) { return -2 * (ax == 0 ? 1 : (ax == 1 ? 3 : 9)) * kPlane; }

// Own pushes of a node pair: f points at node a's slot in plane 0; node b
// sits 4 slabs higher.  xm / xp: the node has an x neighbour inside the block
// on the low / high side.
struct OwnPush {
  float* f;
  bool xm, xp;
  V2 g13;
  template <int J>
  __device__ __forceinline__ void put(V2 v) {
    if constexpr (J == 13) {
      g13 = v;
    } else {
      constexpr int cx = Dir<J>::cx, cy = Dir<J>::cy, cz = Dir<J>::cz;
      constexpr int off = J * kPlane + cx + kPY * cy + kPZ * cz;
      if (cx == 0 || (cx > 0 ? xp : xm)) {
        f[off] = v.v.x;
        f[off + 4 * kPZ] = v.v.y;
      }
    }
  }
};

// Halo pushes in a canonical orientation: the halo node lies just below the
// block on the face axis AX and pushes the 9 directions whose component on
// that axis is +1.  Threads on the upper face reflect their values along the
// face axis first (Eq. three_order_f is covariant under reflections), so
// canonical direction J carries the population of its mirror image, whose
// plane lies mirror_shift(AX) lower.  fa / fb point at the slot, in plane 0
// shifted by the reflection, of the destination of the direction with zero
// components off AX; oka / okb: bit J set when direction J of node a / b
// lands inside the block and has a valid source.
template <int AX>
struct HaloPush {
  float *fa, *fb;
  unsigned oka, okb;
  template <int J>
  __device__ __forceinline__ void put(V2 v) {
    constexpr int cx = Dir<J>::cx, cy = Dir<J>::cy, cz = Dir<J>::cz;
    constexpr int c = AX == 0 ? cx : (AX == 1 ? cy : cz);
    if constexpr (c == 1) {
      constexpr int off = J * kPlane + (AX == 0 ? 0 : cx) + (AX == 1 ? 0 : kPY * cy) + (AX == 2 ? 0 : kPZ * cz);
      if ((oka >> J) & 1u) fa[off] = v.v.x;
      if ((okb >> J) & 1u) fb[off] = v.v.y;
    }
  }
};

// Half-way bounce-back: bit k of mlo / mhi set when the pull source x - c_k of
// node a / b is a wall or a solid node, so slot k of the node receives its own
// population opp(k).  f as in OwnPush.
struct BouncePush {
  float* f;
  unsigned mlo, mhi;
  template <int J>
  __device__ __forceinline__ void put(V2 v) {
    if constexpr (J != 13) {
      constexpr int K = 26 - J;
      if ((mlo >> K) & 1u) f[K * kPlane] = v.v.x;
      if ((mhi >> K) & 1u) f[K * kPlane + 4 * kPZ] = v.v.y;
    }
  }
};

template <int J>
__device__ __forceinline__ void gather_one(const float* f, V2 g13, V2 (&g)[27]) {
  if constexpr (J == 13)
    g[13] = g13;
  else
    g[J] = V2(f[J * kPlane], f[J * kPlane + 4 * kPZ]);
}

// The 27 values of node pair (f as in OwnPush); the rest value comes from g13.
template <int... Js>
__device__ __forceinline__ void gather_all(const float* f, V2 g13, V2 (&g)[27], std::integer_sequence<int, Js...>) {
  (gather_one<Js>(f, g13, g), ...);
}

__host__ __device__ __forceinline__ unsigned range_mask(int v) {
  // bit (c+1) set when v + c lies in [0, 8), c in {-1, 0, 1}
  return ((unsigned)(v - 1) < 8u ? 1u : 0u) | ((unsigned)v < 8u ? 2u : 0u) | ((unsigned)(v + 1) < 8u ? 4u : 0u);
}

// Bit j = (cx+1) + 3 (cy+1) + 9 (cz+1) set when bit cx+1 of vx, bit cy+1 of vy
// and bit cz+1 of vz are all set (per-axis masks as from range_mask).
__host__ __device__ __forceinline__ unsigned dir_mask(unsigned vx, unsigned vy, unsigned vz) {
  const unsigned mx = vx * 0x1249249u;  // vx in every 3-bit group
  const unsigned my = ((vy & 1u) * 0x7u | ((vy >> 1) & 1u) * 0x38u | ((vy >> 2) & 1u) * 0x1C0u) * 0x40201u;
  const unsigned mz = (vz & 1u) * 0x1FFu | ((vz >> 1) & 1u) * 0x3FE00u | ((vz >> 2) & 1u) * 0x7FC0000u;
  return mx & my & mz;
}

// Halo work of thread t < kHaloPairs: cls 0 = x faces (threads 0-63), 1 = y
// faces (64-143), 2 = z faces (144-243), so that only one warp mixes two
// classes; mir = upper face.  Node pair a = (ax, ay, az), b = (bx, by, bz).
__host__ __device__ __forceinline__ void halo_pair(int t, int& cls, bool& mir, int& ax, int& ay, int& az, int& bx, int& by,
                                          int& bz) {
  if (t < 64) {
    const int q = t & 31;
    cls = 0;
    mir = t >= 32;
    ax = bx = mir ? 8 : -1;
    ay = by = q & 7;
    az = q >> 3;
    bz = az + 4;
  } else if (t < 144) {
    const int q = t < 104 ? t - 64 : t - 104;
    cls = 1;
    mir = t >= 104;
    ax = bx = q % 10 - 1;
    ay = by = mir ? 8 : -1;
    az = q / 10;
    bz = az + 4;
  } else {
    const int q = t < 194 ? t - 144 : t - 194;
    cls = 2;
    mir = t >= 194;
    ax = bx = q % 10 - 1;
    ay = q / 10 - 1;
    by = ay + 5;
    az = bz = mir ? 8 : -1;
  }
}

__device__ __forceinline__ int block_dir(int hx, int hy, int hz) {
  const int dx = hx < 0 ? -1 : (hx > 7 ? 1 : 0);
  const int dy = hy < 0 ? -1 : (hy > 7 ? 1 : 0);
  const int dz = hz < 0 ? -1 : (hz > 7 ? 1 : 0);
  return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}

// Bit K set when x - c_K of block-local node (x, y, z) lies in a neighbour
// block whose bit is set in miss (bit (dx+1) + 3 (dy+1) + 9 (dz+1)).  Slot K
// of such a node receives no push: it holds whatever the buffer held before.
__device__ __forceinline__ unsigned missing_sources(int x, int y, int z, unsigned miss) {
  unsigned m = 0;
#pragma unroll
  for (int K = 0; K < 27; ++K) {
    const int cx = K % 3 - 1, cy = (K / 3) % 3 - 1, cz = K / 9 - 1;
    if ((miss >> block_dir(x - cx, y - cy, z - cz)) & 1u) m |= 1u << K;
  }
  return m;
}

__device__ __forceinline__ bool touches_missing(int x, int y, int z, unsigned miss) {
  const unsigned mx = 2u | (x == 0 ? 1u : 0u) | (x == 7 ? 4u : 0u);
  const unsigned my = 2u | (y == 0 ? 1u : 0u) | (y == 7 ? 4u : 0u);
  const unsigned mz = 2u | (z == 0 ? 1u : 0u) | (z == 7 ? 4u : 0u);
  unsigned touched = 0;
#pragma unroll
  for (int iz = 0; iz < 3; ++iz)
#pragma unroll
    for (int iy = 0; iy < 3; ++iy)
      if (((mz >> iz) & 1u) && ((my >> iy) & 1u)) touched |= mx << (3 * iy + 9 * iz);
  return (touched & miss) != 0u;
}

__device__ __forceinline__ Mom<V2> pack(const Mom<float>& a, const Mom<float>& b) {
  Mom<V2> m;
  m.drho = V2(a.drho, b.drho);
  m.ux = V2(a.ux, b.ux);
  m.uy = V2(a.uy, b.uy);
  m.uz = V2(a.uz, b.uz);
  m.sxx = V2(a.sxx, b.sxx);
  m.syy = V2(a.syy, b.syy);
  m.szz = V2(a.szz, b.szz);
  m.sxy = V2(a.sxy, b.sxy);
  m.sxz = V2(a.sxz, b.sxz);
  m.syz = V2(a.syz, b.syz);
  return m;
}

__device__ __forceinline__ Mom<V2> select_halves(const Mom<V2>& a, const Mom<V2>& b, bool lo_b, bool hi_b) {
  // per half: b where the flag is set, else a
  auto sel = [&](V2 x, V2 y) { return V2(lo_b ? y.v.x : x.v.x, hi_b ? y.v.y : x.v.y); };
  Mom<V2> r;
  r.drho = sel(a.drho, b.drho);
  r.ux = sel(a.ux, b.ux);
  r.uy = sel(a.uy, b.uy);
  r.uz = sel(a.uz, b.uz);
  r.sxx = sel(a.sxx, b.sxx);
  r.syy = sel(a.syy, b.syy);
  r.szz = sel(a.szz, b.szz);
  r.sxy = sel(a.sxy, b.sxy);
  r.sxz = sel(a.sxz, b.sxz);
  r.syz = sel(a.syz, b.syz);
  return r;
}

__device__ __forceinline__ Mom<V2> zero_pair() {
  Mom<V2> m;
  m.drho = m.ux = m.uy = m.uz = m.sxx = m.syy = m.szz = m.sxy = m.sxz = m.syz = V2(0.f);
  return m;
}

// Thread geometry and block state shared by the phases of one 8^3 block.
struct PairCtx {
  int t, lane, x, y, z0;
  int own;    // pair slot in global storage (nodes own and own + 256 in natural order)
  int own_p;  // node a's slot in plane 0 of the shared buffer
  uint8_t bf;
  bool solid_any;
  V2 g13;     // rest-direction value of the own pair
};

__device__ __forceinline__ PairCtx pair_ctx() {
  PairCtx c;
  c.t = threadIdx.x;
  c.lane = c.t & 31;
  const int w = c.t >> 5;
  c.x = c.lane & 7;
  c.y = (c.lane >> 3) + ((w & 1) << 2);
  c.z0 = w >> 1;
  c.own = c.x + 8 * c.y + 64 * c.z0;
  c.own_p = pidx(c.x, c.y, c.z0);
  return c;
}

// Streaming of one 8^3 block through the destination-indexed shared buffer:
// every node pair emits 27 values (Src::emit) that land at the node the
// value streams to; halo pairs of the 26 neighbour blocks supply the values
// entering the block; bounce-back slots take the node's own value of the
// opposite direction.  Src supplies the node values: lambda_p and its
// transposed projection for the reverse step of the adjoint (the forward
// kernel writes the same phases out for the stored moments).  Ends with a
// barrier; the caller gathers.  Src provides Node, own(blk, slot),
// pair(blk, slot), two(ba, ca, bb, cb), zero(), mirror(node, axis, sign) and
// emit(node, sink).
template <typename Src>
__device__ __forceinline__ void stream_pairs(const Src& src, const StepArgs& a, const int64_t blk, float2* f2buf,
                                             unsigned& s_miss, PairCtx& cx) {
  float* fbuf = reinterpret_cast<float*>(f2buf);
  const int t = cx.t, x = cx.x, own = cx.own;

  if (t < 32) {
    const int v = t < 27 ? a.nbr[blk * 27 + t] : 0;
    const unsigned mb = __ballot_sync(0xffffffffu, t < 27 && is_copy_nbr(v));
    if (t == 0) s_miss = mb;
  }
  const uint8_t bf = a.bflags != nullptr ? a.bflags[blk] : 0;
  const bool solid_any = (bf & kBlockSolidNear) != 0;
  cx.bf = bf;
  cx.solid_any = solid_any;

  // own node pair: issue the loads early
  const typename Src::Node m = src.own(blk, own);
  int cls = -1, hax = 0, hay = 0, haz = 0, hbx = 0, hby = 0, hbz = 0;
  bool mir = false;
  if (t < kHaloPairs) halo_pair(t, cls, mir, hax, hay, haz, hbx, hby, hbz);

  bool va = false, vb = false;
  typename Src::Node hm = Src::zero();
  if (t < kHaloPairs) {
    const int na = __ldg(a.nbr + blk * 27 + block_dir(hax, hay, haz));
    const int nb = __ldg(a.nbr + blk * 27 + block_dir(hbx, hby, hbz));
    const int sa = (hax & 7) + 8 * (hay & 7) + 64 * (haz & 7), sb = (hbx & 7) + 8 * (hby & 7) + 64 * (hbz & 7);
    va = na >= 0 && !(solid_any && a.solid[int64_t(na) * kCells + sa]);
    vb = nb >= 0 && !(solid_any && a.solid[int64_t(nb) * kCells + sb]);
    if (cls < 2) {  // x / y faces: a and b are one stored pair of the same neighbour
      if (na >= 0) hm = src.pair(na, sa);
    } else {
      hm = src.two(na, sa, nb, sb);
    }
  }

  // A. halo pairs (before the own pair: the halo values are then dead before
  // the own pair's are expanded)
  if (t < kHaloPairs && (va || vb)) {
    // reflect the upper-face pairs along the face axis
    Src::mirror(hm, cls, V2(mir ? -1.f : 1.f));
    const unsigned ma = va ? ~0u : 0u, mb = vb ? ~0u : 0u;
    const int dst = mir ? 7 : 0;  // destination coordinate on the face axis
    if (cls == 0) {
      const int sh = mir ? mirror_shift(0) : 0;
      HaloPush<0> s{fbuf + sh + pidx(dst, hay, haz), fbuf + sh + pidx(dst, hby, hbz),
                    dir_mask(7u, range_mask(hay), range_mask(haz)) & ma,
                    dir_mask(7u, range_mask(hby), range_mask(hbz)) & mb};
      src.emit(hm, s);
    } else if (cls == 1) {
      const int sh = mir ? mirror_shift(1) : 0;
      HaloPush<1> s{fbuf + sh + pidx(hax, dst, haz), fbuf + sh + pidx(hbx, dst, hbz),
                    dir_mask(range_mask(hax), 7u, range_mask(haz)) & ma,
                    dir_mask(range_mask(hbx), 7u, range_mask(hbz)) & mb};
      src.emit(hm, s);
    } else {
      const int sh = mir ? mirror_shift(2) : 0;
      HaloPush<2> s{fbuf + sh + pidx(hax, hay, dst), fbuf + sh + pidx(hbx, hby, dst),
                    dir_mask(range_mask(hax), range_mask(hay), 7u) & ma,
                    dir_mask(range_mask(hbx), range_mask(hby), 7u) & mb};
      src.emit(hm, s);
    }
  }

  // B. the own pair, then bounce-back: a solid node of the block also pushed
  // into the slots that bounce-back fills, so blocks with solid nodes order
  // the two writes with a barrier (block-uniform condition)
  float* const fown = fbuf + cx.own_p;
  OwnPush op{fown, x > 0, x < 7, V2(0.f)};
  src.emit(m, op);
  cx.g13 = op.g13;
  if (bf & kBlockBounce) {
    if (solid_any) __syncthreads();
    const unsigned mlo_b = a.bmask[blk * kCells + own], mhi_b = a.bmask[blk * kCells + own + 256];
    if ((mlo_b | mhi_b) != 0u) {
      BouncePush bp{fown, mlo_b, mhi_b};
      src.emit(src.own(blk, own), bp);
    }
  }
  __syncthreads();
}

}  // namespace f2
}  // namespace hlbm
