// stream_collide_f2.cu -- FP32-math stream-collide for FP32 and reduced-precision
// storage: two nodes per thread with packed FP32 arithmetic.
//
// One CTA per stored 8^3 block, 256 threads.  Thread (lane, warp) owns the node
// pair (x, y, z0) and (x, y, z0 + 4) with x = lane & 7, y = (lane >> 3) + 4 (warp & 1),
// z0 = warp >> 1.  Shared memory holds, per direction j, the pulled population
// of every node of the block, destination-indexed, in a padded plane: node
// (x, y, z) at x + 8 (y + 1) + kPZ (z + 1), with rows y = -1, 8 and slabs
// z = -1, 8 as padding that is written but never read (and shared between
// neighbouring rows, slabs and planes).  Every store of a node
// is then at a compile-time offset from one base address per node, and the
// 32 lanes of a warp touch 32 consecutive words (no bank conflicts for the
// own pushes and the gather).  Each (destination, direction) slot has exactly
// one writer, so the pushes need no ordering among themselves:
//  A. 244 threads each take a pair of halo nodes (read from the 26 neighbour
//     blocks, mostly L2 hits) and write the 9 directions that enter the block
//     (one code path per face axis: upper faces are reflected onto lower
//     ones, which shifts the store by a whole number of planes);
//  B. each thread reconstructs the 26 moving populations of its pair
//     (Eq. three_order_f) and pushes them to their destinations x + c_j
//     (pushes through an x face are predicated off, those through a y or z
//     face land in the padding); nodes whose pull source is a wall or a solid
//     node write their own opposite population instead (half-way
//     bounce-back; after a barrier in blocks with solid nodes, whose own
//     pushes that slot also receives);
//  C. after one barrier, each thread reads the 26 populations of its pair,
//     projects to moments (Eq. rho_u_stress) and collides (Sec. 3.1; Guo
//     forcing; mixture tau of Sec. 4).  Interface nodes (a neighbour block not
//     stored) and solid nodes copy their input.
// Modes: kPlain; kRecord also writes the pre-collision moments (recomputed
// steps of the adjoint); kStreamOnly writes them instead of colliding (the
// streaming-only step S of a coupled step, Fig. 4; the collision follows
// once the drag has been exchanged).
#include <utility>

#include "f2_common.cuh"
#include "hlbm_internal.h"
#include "lbm_math.cuh"
#include "v2.cuh"

namespace hlbm {
namespace {

using namespace f2;

// Geometric direction masks (node a, node b) of halo pair t: bit J set when
// canonical direction J of that node lands inside the block.  They depend on
// t only, so the host computes them once with the functions the halo phase
// would use (one 8-byte load per halo thread instead of the mask arithmetic).
__device__ uint2 g_halo_masks[kHaloPairs];

void halo_masks_host(uint2* out) {
  for (int t = 0; t < kHaloPairs; ++t) {
    int cls, hax, hay, haz, hbx, hby, hbz;
    bool mir;
    halo_pair(t, cls, mir, hax, hay, haz, hbx, hby, hbz);
    unsigned a, b;
    if (cls == 0) {
      a = dir_mask(7u, range_mask(hay), range_mask(haz));
      b = dir_mask(7u, range_mask(hay), range_mask(hbz));
    } else if (cls == 1) {
      a = dir_mask(range_mask(hax), 7u, range_mask(haz));
      b = dir_mask(range_mask(hax), 7u, range_mask(hbz));
    } else {
      a = dir_mask(range_mask(hax), range_mask(hay), 7u);
      b = dir_mask(range_mask(hax), range_mask(hby), 7u);
    }
    out[t] = make_uint2(a, b);
  }
}

// Upload the masks to the current device once.
cudaError_t ensure_halo_masks() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  uint2 h[kHaloPairs];
  halo_masks_host(h);
  e = cudaMemcpyToSymbol(g_halo_masks, h, sizeof(h));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

// One 8^3 block of the forward step: push the own and halo populations into
// the destination-indexed shared buffer, then gather, project and collide.
// Leaves shared memory in use: callers that process another block must
// barrier first.  The streaming phases are the ones of f2::stream_pairs
// (which the reverse step of the adjoint instantiates) written out for the
// moment source: this form measured 2 % faster for the forward kernel.
enum ScMode { kPlain = 0, kRecord = 1, kStreamOnly = 2 };

template <typename T, int kMode = kPlain>
__device__ __forceinline__ void sc_block(const StepArgs& a, const int64_t blk, float2* f2buf, unsigned& s_miss) {
  float* fbuf = reinterpret_cast<float*>(f2buf);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int x = lane & 7, y = (lane >> 3) + ((w & 1) << 2), z0 = w >> 1;
  const int own = x + 8 * y + 64 * z0;                 // pair slot in global storage
  const T* in = static_cast<const T*>(a.in);
  T* out = static_cast<T*>(a.out);
  const int dom = a.blk_dom != nullptr ? a.blk_dom[blk] : 0;
  const Scales* sc_in = a.scales_in != nullptr ? a.scales_in + dom : nullptr;
  const Scales* sc_out = a.scales_out != nullptr ? a.scales_out + dom : nullptr;

  // missing neighbours (interface nodes): read in phase C, after the barriers
  if (t < 32) {
    const int v = t < 27 ? a.nbr[blk * 27 + t] : 0;
    const unsigned mb = __ballot_sync(0xffffffffu, t < 27 && is_copy_nbr(v));
    if (t == 0) s_miss = mb;
  }
  const uint8_t bf = a.bflags != nullptr ? a.bflags[blk] : 0;
  const bool solid_any = (bf & kBlockSolidNear) != 0;

  // own node pair: issue the loads early
  const Mom<V2> m = load_pair<T>(in, blk, own, sc_in);
  int cls = -1, hax = 0, hay = 0, haz = 0, hbx = 0, hby = 0, hbz = 0;
  bool mir = false;
  if (t < kHaloPairs) halo_pair(t, cls, mir, hax, hay, haz, hbx, hby, hbz);

  // halo pairs: each thread reads its two neighbour entries itself, so no
  // barrier waits for the table (measured 7 % faster than sharing it)
  // a halo node without a stored neighbour reads the block's own node at the
  // same slot instead (finite values whose pushes the masks drop), so the
  // loads need no branch and no zeroing
  bool va = false, vb = false;
  Mom<V2> hm;
  if (t < kHaloPairs) {
    const int na = __ldg(a.nbr + blk * 27 + block_dir(hax, hay, haz));
    const int nb = __ldg(a.nbr + blk * 27 + block_dir(hbx, hby, hbz));
    const int sa = (hax & 7) + 8 * (hay & 7) + 64 * (haz & 7), sb = (hbx & 7) + 8 * (hby & 7) + 64 * (hbz & 7);
    va = na >= 0 && !(solid_any && a.solid[int64_t(na) * kCells + sa]);
    vb = nb >= 0 && !(solid_any && a.solid[int64_t(nb) * kCells + sb]);
    const int64_t ba = na >= 0 ? int64_t(na) : blk, bb = nb >= 0 ? int64_t(nb) : blk;
    if (cls < 2)  // x / y faces: a and b are one stored pair of the same neighbour
      hm = load_pair<T>(in, ba, sa, sc_in);
    else
      hm = pack(load_node<T>(in, ba, sa, sc_in), load_node<T>(in, bb, sb, sc_in));
  }

  const V2 kxyz = V2(a.kxyzf);
  // A. halo pairs
  if (t < kHaloPairs && (va || vb)) {
    // reflect the upper-face pairs along the face axis (u and S components with
    // an odd count of that axis change sign)
    const V2 sg = V2(mir ? -1.f : 1.f);
    if (cls == 0) {
      hm.ux = hm.ux * sg;
      hm.sxy = hm.sxy * sg;
      hm.sxz = hm.sxz * sg;
    } else if (cls == 1) {
      hm.uy = hm.uy * sg;
      hm.sxy = hm.sxy * sg;
      hm.syz = hm.syz * sg;
    } else {
      hm.uz = hm.uz * sg;
      hm.sxz = hm.sxz * sg;
      hm.syz = hm.syz * sg;
    }
    const Coef<V2> c = make_coef(hm, kxyz);
    const unsigned ma = va ? ~0u : 0u, mb = vb ? ~0u : 0u;
    const uint2 gm = g_halo_masks[t];
    const int dst = mir ? 7 : 0;  // destination coordinate on the face axis
    if (cls == 0) {
      const int sh = mir ? mirror_shift(0) : 0;
      HaloPush<0> hp{fbuf + sh + pidx(dst, hay, haz), fbuf + sh + pidx(dst, hby, hbz), gm.x & ma, gm.y & mb};
      emit_all(c, hp);
    } else if (cls == 1) {
      const int sh = mir ? mirror_shift(1) : 0;
      HaloPush<1> hp{fbuf + sh + pidx(hax, dst, haz), fbuf + sh + pidx(hbx, dst, hbz), gm.x & ma, gm.y & mb};
      emit_all(c, hp);
    } else {
      const int sh = mir ? mirror_shift(2) : 0;
      HaloPush<2> hp{fbuf + sh + pidx(hax, hay, dst), fbuf + sh + pidx(hbx, hby, dst), gm.x & ma, gm.y & mb};
      emit_all(c, hp);
    }
  }
  // B. push the own pair (after the halo pairs: the halo moments are then
  // dead before the own coefficients are formed, 106 instead of 128 registers
  // in FP32)
  float* const fown = fbuf + pidx(x, y, z0);
  OwnPush op{fown, x > 0, x < 7, V2(0.f)};
  emit_all(make_coef(m, kxyz), op);

  // bounce-back: a solid node of the block also pushed into the slots it
  // fills, so blocks with solid nodes order the two writes with a barrier
  // (block-uniform condition)
  if (bf & kBlockBounce) {
    if (solid_any) __syncthreads();
    const unsigned mlo_b = a.bmask[blk * kCells + own], mhi_b = a.bmask[blk * kCells + own + 256];
    if ((mlo_b | mhi_b) != 0u) {
      BouncePush bp{fown, mlo_b, mhi_b};
      emit_all(make_coef(load_pair<T>(in, blk, own, sc_in), kxyz), bp);
    }
  }
  __syncthreads();

  // C. gather, project, collide
  bool copy_lo = false, copy_hi = false;
  if (solid_any) {
    copy_lo = a.solid[blk * kCells + own] != 0;
    copy_hi = a.solid[blk * kCells + own + 256] != 0;
  }
  if (s_miss != 0u) {
    copy_lo = copy_lo || touches_missing(x, y, z0, s_miss);
    copy_hi = copy_hi || touches_missing(x, y, z0 + 4, s_miss);
  }
  Mom<V2> mo;
  if constexpr (kMode == kStreamOnly) {  // the collision step copies the input at these nodes
    if (copy_lo && copy_hi) return;
  }
  if (copy_lo && copy_hi) {
    mo = load_pair<T>(in, blk, own, sc_in);
  } else {
    V2 g[27];
    gather_all(fown, op.g13, g, std::make_integer_sequence<int, 27>{});
    const PreMom<V2> p = project(g);
    if constexpr (kMode != kPlain) {  // pre-collision moments (natural order, float32)
      float* q = a.pre_out + blk * (kRows * kCells) + own;
      const V2 r[kRows] = {p.drho, p.jx, p.jy, p.jz, p.pxx, p.pyy, p.pzz, p.pxy, p.pxz, p.pyz};
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        q[k * kCells] = r[k].v.x;
        q[k * kCells + 256] = r[k].v.y;
      }
      if constexpr (kMode == kStreamOnly) return;
    }
    V2 fx, fy, fz;
    if (a.F != nullptr) {
      const float* Fp = a.F + blk * 3 * kCells + own;
      fx = V2(__ldg(Fp), __ldg(Fp + 256));
      fy = V2(__ldg(Fp + kCells), __ldg(Fp + kCells + 256));
      fz = V2(__ldg(Fp + 2 * kCells), __ldg(Fp + 2 * kCells + 256));
    } else {
      fx = V2(a.fuf[0]);
      fy = V2(a.fuf[1]);
      fz = V2(a.fuf[2]);
    }
    V2 om = V2(a.blk_om != nullptr ? __ldg(a.blk_om + blk) : a.omf);
    if (a.eps != nullptr)
      om = inv(V2(a.tauf) * V2(__ldg(a.eps + blk * kCells + own), __ldg(a.eps + blk * kCells + own + 256)));
    mo = collide(p, fx, fy, fz, om);
    if (copy_lo || copy_hi) mo = select_halves(mo, load_pair<T>(in, blk, own, sc_in), copy_lo, copy_hi);
  }
  store_pair<T>(out, blk, own, mo, sc_out);
}

// One CTA per block.
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_stream_collide_f2(StepArgs a) {
  extern __shared__ __align__(16) float2 f2buf[];  // padded planes, kBufBytes
  __shared__ unsigned s_miss;
  sc_block<T>(a, a.blk0 + blockIdx.x, f2buf, s_miss);
}

// The same step, also writing the pre-collision moments to a.pre_out (the
// recomputed forward steps of the adjoint).
__global__ void __launch_bounds__(kThreads, 2) k_stream_collide_f2_record(StepArgs a) {
  extern __shared__ __align__(16) float2 f2buf[];
  __shared__ unsigned s_miss;
  sc_block<float, kRecord>(a, a.blk0 + blockIdx.x, f2buf, s_miss);
}

// The streaming-only step: pre-collision moments to a.pre_out, no collision.
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_stream_f2_pre(StepArgs a) {
  extern __shared__ __align__(16) float2 f2buf[];
  __shared__ unsigned s_miss;
  sc_block<T, kStreamOnly>(a, a.blk0 + blockIdx.x, f2buf, s_miss);
}

// Persistent CTAs (a grid sized to the resident capacity) that take blocks
// from an atomic ticket counter in list order.  work[0] is the ticket counter,
// work[1] counts finished CTAs; the last CTA to finish puts both back to zero
// for the next launch on the stream.  No CTA waits on another.
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_stream_collide_f2_persistent(StepArgs a) {
  extern __shared__ __align__(16) float2 f2buf[];
  __shared__ unsigned s_miss;
  __shared__ unsigned s_tk;
  unsigned* work = a.work;
  if (threadIdx.x == 0) s_tk = atomicAdd(work, 1u);
  __syncthreads();
  unsigned tk = s_tk;
  while (tk < unsigned(a.nb)) {
    sc_block<T>(a, a.blk0 + tk, f2buf, s_miss);
    __syncthreads();  // shared buffers free again
    if (threadIdx.x == 0) s_tk = atomicAdd(work, 1u);
    __syncthreads();
    tk = s_tk;
  }
  if (threadIdx.x == 0) {
    // every CTA that reaches this point has taken its last ticket
    __threadfence();
    if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {
      work[0] = 0u;
      work[1] = 0u;
    }
  }
}

// Per-node bounce masks: bit k set when the pull source x - c_k of node x is
// beyond a wall or a solid node.  Sets kBlockBounce on blocks with any bit.
__global__ void __launch_bounds__(512) k_bounce_masks(const int32_t* __restrict__ nbr,
                                                      const uint8_t* __restrict__ solid, uint8_t* __restrict__ bflags,
                                                      uint32_t* __restrict__ bmask) {
  const int64_t blk = blockIdx.x;
  const int n = threadIdx.x;
  const int x = n & 7, y = (n >> 3) & 7, z = n >> 6;
  const bool solid_any = solid != nullptr && (bflags[blk] & kBlockSolidNear);
  // no wall among the 26 neighbours and no solid nearby: no bounce-back (the
  // masks of such blocks are never read)
  __shared__ int s_wall;
  if (n == 0) s_wall = 0;
  __syncthreads();
  if (n < 27 && nbr[blk * 27 + n] == kWall) s_wall = 1;
  __syncthreads();
  if (!s_wall && !solid_any) {
    if (n == 0) bflags[blk] = uint8_t(bflags[blk] & ~kBlockBounce);
    return;
  }
  unsigned m = 0;
  for (int k = 0; k < 27; ++k) {
    if (k == 13) continue;
    const int sx = x - (k % 3 - 1), sy = y - ((k / 3) % 3 - 1), sz = z - (k / 9 - 1);
    const int dx = sx < 0 ? -1 : (sx > 7 ? 1 : 0), dy = sy < 0 ? -1 : (sy > 7 ? 1 : 0),
              dz = sz < 0 ? -1 : (sz > 7 ? 1 : 0);
    const int32_t q = nbr[blk * 27 + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
    bool hit = q == kWall;
    if (!hit && solid_any && q >= 0) hit = solid[int64_t(q) * kCells + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7)] != 0;
    if (hit) m |= 1u << k;
  }
  bmask[blk * kCells + n] = m;
  const int any = __syncthreads_or(m != 0u);
  if (n == 0) bflags[blk] = uint8_t((bflags[blk] & ~kBlockBounce) | (any ? kBlockBounce : 0));
}

template <typename T>
cudaError_t launch_f2(const StepArgs& a_in, cudaStream_t s) {
  {
    const cudaError_t e = ensure_halo_masks();
    if (e != cudaSuccess) return e;
  }
  StepArgs a = a_in;
  for (int k = 0; k < 3; ++k) a.fuf[k] = float(a.fu[k]);
  a.tauf = float(a.tau);
  a.omf = float(a.om);
  a.kxyzf = float(a.kxyz);
  const size_t smem = kBufBytes;
  static bool configured = false;
  if (!configured) {
    cudaError_t err =
        cudaFuncSetAttribute(k_stream_collide_f2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_stream_collide_f2_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (err != cudaSuccess) return err;
    configured = true;
  }
  if (a.nb == 0) return cudaSuccess;
  if (a.work != nullptr) {
    if (a.grid <= 0 || a.nb >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
    k_stream_collide_f2_persistent<T><<<unsigned(a.grid), kThreads, smem, s>>>(a);
  } else {
    k_stream_collide_f2<T><<<(unsigned)a.nb, kThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t resident_f2(int* per_sm) {
  const size_t smem = kBufBytes;
  cudaError_t err =
      cudaFuncSetAttribute(k_stream_collide_f2_persistent<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_stream_collide_f2_persistent<T>, kThreads, smem);
}

}  // namespace

cudaError_t launch_stream_collide_f2(int storage, const StepArgs& a, cudaStream_t s) {
  switch (storage) {
    case HLBM_STORE_F32: return launch_f2<float>(a, s);
    case HLBM_STORE_F16S: return launch_f2<__half>(a, s);
    case HLBM_STORE_BF16S: return launch_f2<__nv_bfloat16>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stream_collide_record(const StepArgs& a_in, cudaStream_t s) {
  {
    const cudaError_t e = ensure_halo_masks();
    if (e != cudaSuccess) return e;
  }
  StepArgs a = a_in;
  for (int k = 0; k < 3; ++k) a.fuf[k] = float(a.fu[k]);
  a.tauf = float(a.tau);
  a.omf = float(a.om);
  a.kxyzf = float(a.kxyz);
  const size_t smem = kBufBytes;
  static bool configured = false;
  if (!configured) {
    cudaError_t err =
        cudaFuncSetAttribute(k_stream_collide_f2_record, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    configured = true;
  }
  if (a.nb == 0) return cudaSuccess;
  if (a.pre_out == nullptr) return cudaErrorInvalidValue;
  k_stream_collide_f2_record<<<(unsigned)a.nb, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pre(const StepArgs& a_in, cudaStream_t s) {
  {
    const cudaError_t e = ensure_halo_masks();
    if (e != cudaSuccess) return e;
  }
  StepArgs a = a_in;
  const size_t smem = kBufBytes;
  static bool configured = false;
  if (!configured) {
    cudaError_t err =
        cudaFuncSetAttribute(k_stream_f2_pre<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    configured = true;
  }
  for (int k = 0; k < 3; ++k) a.fuf[k] = float(a.fu[k]);
  a.tauf = float(a.tau);
  a.omf = float(a.om);
  a.kxyzf = float(a.kxyz);
  if (a.nb == 0) return cudaSuccess;
  if (a.pre_out == nullptr) return cudaErrorInvalidValue;
  k_stream_f2_pre<T><<<(unsigned)a.nb, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stream_only(int storage, const StepArgs& a, cudaStream_t s) {
  switch (storage) {
    case HLBM_STORE_F32: return launch_pre<float>(a, s);
    case HLBM_STORE_F16S: return launch_pre<__half>(a, s);
    case HLBM_STORE_BF16S: return launch_pre<__nv_bfloat16>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t persistent_ctas_per_sm(int storage, int* per_sm) {
  switch (storage) {
    case HLBM_STORE_F32: return resident_f2<float>(per_sm);
    case HLBM_STORE_F16S: return resident_f2<__half>(per_sm);
    case HLBM_STORE_BF16S: return resident_f2<__nv_bfloat16>(per_sm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t compute_bounce_masks(const int32_t* nbr, const uint8_t* solid, uint8_t* bflags, uint32_t* bmask, int64_t nb,
                                 cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  k_bounce_masks<<<unsigned(nb), 512, 0, s>>>(nbr, solid, bflags, bmask);
  return cudaGetLastError();
}

}  // namespace hlbm
