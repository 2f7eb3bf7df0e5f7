// f2_common.cuh -- building blocks of the node-pair kernels (FP32 math on
// packed pairs of nodes (z, z + 4) of an 8^3 block, 256 threads per block):
// the destination-indexed shared population buffer and its pushes (own pairs,
// halo pairs reflected onto the lower face of each axis, bounce-back), the
// gather, and the assignment of halo pairs to threads.  Used by the forward
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

__host__ __device__ constexpr int slot_of(int j) { return j < 13 ? j : j - 1; }

struct OwnPush {
  float2* f;
  int XH[9], Y8[3], Z64[3];  // XH[(cx+1) + 3 (cy+1)] = x' ^ (y' >> 1)
  bool swap[3];
  V2 g13;
  template <int J>
  __device__ __forceinline__ void put(V2 v) {
    if constexpr (J == 13) {
      g13 = v;
    } else {
      constexpr int cx = Dir<J>::cx, cy = Dir<J>::cy, cz = Dir<J>::cz;
      const int s = XH[(cx + 1) + 3 * (cy + 1)] + Y8[cy + 1] + Z64[cz + 1];
      f[slot_of(J) * 256 + s] = swap[cz + 1] ? make_float2(v.v.y, v.v.x) : v.v;
    }
  }
};

constexpr int kTrash = 26 * 512;  // per-lane dummy float slots for masked halo stores

// Halo pushes in a canonical orientation: the halo node lies just below the
// block on the face axis and pushes the 9 directions whose component on that
// axis is +1.  Threads on the upper face reflect their moments along the face
// axis first (Eq. three_order_f is covariant under reflections), so canonical
// direction J carries the population of its mirror image; d0 / d1 shift the
// store to the mirror direction's slot (d1 for the mirrors that lie on the
// other side of the rest index).  oka / okb: bit J set when the .x / .y value
// of canonical direction J has a destination inside the block and a valid
// source; other values go to the lane's trash slot.

// x faces (AX = 0) and y faces (AX = 1): node pair a = (hx, hy, hz), b = hz + 4,
// one stored pair of the same neighbour.  X / YH / Y8 / Z64 hold the actual
// destination coordinates (swizzle parts) for canonical component c at [c+1];
// ha[c+1]: node a lands in the high half of its pair slot.
template <int AX>
struct HaloXY {
  float* f;
  int X[3], YH[3], Y8[3], Z64[3], ha[3];
  unsigned oka, okb;
  int d0, d1, trash;
  template <int J>
  __device__ __forceinline__ void put(V2 v) {
    constexpr int cx = Dir<J>::cx, cy = Dir<J>::cy, cz = Dir<J>::cz;
    constexpr int c = AX == 0 ? cx : cy;
    if constexpr (c == 1) {
      constexpr bool cross = AX == 0 ? (cy == 0 && cz == 0) : (cz == 0);
      const int p2 = 2 * (slot_of(J) * 256 + (X[cx + 1] ^ YH[cy + 1]) + Y8[cy + 1] + Z64[cz + 1]) + (cross ? d1 : d0);
      const int h = ha[cz + 1];
      f[((oka >> J) & 1u) ? p2 + h : trash] = v.v.x;
      f[((okb >> J) & 1u) ? p2 + 1 - h : trash] = v.v.y;
    }
  }
};

// z faces: node pair a = (hx, hy, hz), b = (hx, hy + 5, hz); zoff addresses the
// destination plane (z = 0: pair slot 0, low half; z = 7: pair slot 3, high half).
struct HaloZ {
  float* f;
  int X[3], YHa[3], YHb[3], Y8a[3], Y8b[3];
  int zoff;
  unsigned oka, okb;
  int d, trash;
  template <int J>
  __device__ __forceinline__ void put(V2 v) {
    constexpr int cx = Dir<J>::cx, cy = Dir<J>::cy, cz = Dir<J>::cz;
    if constexpr (cz == 1) {
      const int base = 2 * (slot_of(J) * 256) + zoff + d;
      f[((oka >> J) & 1u) ? base + 2 * ((X[cx + 1] ^ YHa[cy + 1]) + Y8a[cy + 1]) : trash] = v.v.x;
      f[((okb >> J) & 1u) ? base + 2 * ((X[cx + 1] ^ YHb[cy + 1]) + Y8b[cy + 1]) : trash] = v.v.y;
    }
  }
};

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

// Half-way bounce-back: bit k of mask = the pull source x - c_k of this node is
// a wall or a solid node, so slot k of the node receives its own population opp(k).
struct BouncePush {
  float* f;
  int own;  // pair slot
  unsigned mlo, mhi;
  template <int J>
  __device__ __forceinline__ void put(V2 v) {
    if constexpr (J != 13) {
      constexpr int K = 26 - J;
      if ((mlo >> K) & 1u) f[2 * (slot_of(K) * 256 + own)] = v.v.x;
      if ((mhi >> K) & 1u) f[2 * (slot_of(K) * 256 + own) + 1] = v.v.y;
    }
  }
};

template <int J>
__device__ __forceinline__ void gather_one(const float2* f, int own, V2 g13, V2 (&g)[27]) {
  if constexpr (J == 13)
    g[13] = g13;
  else
    g[J] = V2(f[slot_of(J) * 256 + own]);
}

template <int... Js>
__device__ __forceinline__ void gather_all(const float2* f, int own, V2 g13, V2 (&g)[27],
                                           std::integer_sequence<int, Js...>) {
  (gather_one<Js>(f, own, g13, g), ...);
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
// of such a node receives no halo push: it still holds a wrapped own push.
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
  int own_s;  // pair slot in shared memory
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
  c.own_s = (c.x ^ (c.y >> 1)) + 8 * c.y + 64 * c.z0;
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
  const int t = cx.t, lane = cx.lane, x = cx.x, y = cx.y, z0 = cx.z0, own = cx.own, own_s = cx.own_s;

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

  // A. push the own pair
  OwnPush op;
  op.f = f2buf;
#pragma unroll
  for (int c = -1; c <= 1; ++c) {
    op.Y8[c + 1] = 8 * ((y + c) & 7);
    op.Z64[c + 1] = 64 * ((z0 + c) & 3);
    op.swap[c + 1] = (((z0 + c) & 7) >> 2) != 0;
#pragma unroll
    for (int cx = -1; cx <= 1; ++cx) op.XH[(cx + 1) + 3 * (c + 1)] = ((x + cx) & 7) ^ (((y + c) & 7) >> 1);
  }
  src.emit(m, op);
  cx.g13 = op.g13;
  __syncthreads();

  // B. halo pairs and bounce-back
  if (t < kHaloPairs && (va || vb)) {
    // reflect the upper-face pairs along the face axis
    Src::mirror(hm, cls, V2(mir ? -1.f : 1.f));
    const int trash = kTrash + lane;
    const unsigned ma = va ? ~0u : 0u, mb = vb ? ~0u : 0u;
    if (cls < 2) {
      int Zc[3], HA[3];
#pragma unroll
      for (int k = -1; k <= 1; ++k) {
        Zc[k + 1] = 64 * ((haz + k) & 3);
        HA[k + 1] = ((haz + k) & 7) >> 2;
      }
      const unsigned vza = range_mask(haz), vzb = range_mask(hbz);
      const int face_dst = mir ? 7 : 0;  // destination coordinate on the face axis
      if (cls == 0) {
        int YH[3], Y8[3];
#pragma unroll
        for (int k = -1; k <= 1; ++k) {
          YH[k + 1] = ((hay + k) & 7) >> 1;
          Y8[k + 1] = 8 * ((hay + k) & 7);
        }
        const unsigned vy = range_mask(hay);
        HaloXY<0> s{fbuf, {0, 0, face_dst}, {YH[0], YH[1], YH[2]}, {Y8[0], Y8[1], Y8[2]}, {Zc[0], Zc[1], Zc[2]},
                    {HA[0], HA[1], HA[2]}, dir_mask(7u, vy, vza) & ma, dir_mask(7u, vy, vzb) & mb,
                    mir ? -1024 : 0, mir ? -512 : 0, trash};
        src.emit(hm, s);
      } else {
        int X[3];
#pragma unroll
        for (int k = -1; k <= 1; ++k) X[k + 1] = (hax + k) & 7;
        const unsigned vx = range_mask(hax);
        HaloXY<1> s{fbuf, {X[0], X[1], X[2]}, {0, 0, face_dst >> 1}, {0, 0, 8 * face_dst}, {Zc[0], Zc[1], Zc[2]},
                    {HA[0], HA[1], HA[2]}, dir_mask(vx, 7u, vza) & ma, dir_mask(vx, 7u, vzb) & mb,
                    mir ? -3072 : 0, mir ? -2560 : 0, trash};
        src.emit(hm, s);
      }
    } else {
      int X[3], YHa[3], YHb[3], Y8a[3], Y8b[3];
#pragma unroll
      for (int k = -1; k <= 1; ++k) {
        X[k + 1] = (hax + k) & 7;
        YHa[k + 1] = ((hay + k) & 7) >> 1;
        YHb[k + 1] = ((hby + k) & 7) >> 1;
        Y8a[k + 1] = 8 * ((hay + k) & 7);
        Y8b[k + 1] = 8 * ((hby + k) & 7);
      }
      const unsigned vx = range_mask(hax);
      HaloZ s{fbuf, {X[0], X[1], X[2]}, {YHa[0], YHa[1], YHa[2]}, {YHb[0], YHb[1], YHb[2]},
              {Y8a[0], Y8a[1], Y8a[2]}, {Y8b[0], Y8b[1], Y8b[2]}, mir ? 2 * 64 * 3 + 1 : 0,
              dir_mask(vx, range_mask(hay), 7u) & ma, dir_mask(vx, range_mask(hby), 7u) & mb, mir ? -17 * 512 : 0,
              trash};
      src.emit(hm, s);
    }
  }
  if (bf & kBlockBounce) {  // block-uniform
    const unsigned mlo_b = a.bmask[blk * kCells + own], mhi_b = a.bmask[blk * kCells + own + 256];
    if ((mlo_b | mhi_b) != 0u) {
      BouncePush bp{fbuf, own_s, mlo_b, mhi_b};
      src.emit(src.own(blk, own), bp);
    }
  }
  __syncthreads();
}

}  // namespace f2
}  // namespace hlbm
