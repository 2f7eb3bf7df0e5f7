// storage.cuh -- moment storage policies.
//
// A level's moments live block-major as [n_blocks][10 rows][512 nodes] in one of:
//   double  (80 B/node), float (40 B/node),
//   half / bf16 with a per-row power-of-two scale (20 B/node).
// Row 0 holds delta_rho = rho - 1 for every policy.  The reduced-precision
// policies hold delta_rho, u and S^neq = S - u u, each times 2^e_r with one
// exponent per row and level (the scale is exact, so decoding is
// value = code * 2^-e_r); all their arithmetic is done in float.
//
// Node order inside a row: double keeps the natural order x + 8 y + 64 z.  The
// FP32-math policies (float, half, bf16) interleave the node pair (x, y, z) and
// (x, y, z + 4) for z < 4: node (x, y, z) sits at 2 (x + 8 y + 64 (z & 3)) + (z >> 2),
// so the pair a thread of the packed-FP32 kernel owns is one 64-bit word.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "lbm_math.cuh"
#include "v2.cuh"

namespace hlbm {

constexpr int kRows = 10;
constexpr int kCells = 512;

struct Scales {
  float enc[kRows];  // 2^e_r
  float dec[kRows];  // 2^-e_r
};

template <typename T>
struct StorageTraits;

template <>
struct StorageTraits<double> {
  using R = double;
  static constexpr bool kNeq = false;
  static constexpr bool kPaired = false;
  __device__ static R load(const double* p) { return __ldg(p); }
  __device__ static void store(double* p, R v) { __stcs(p, v); }
};

template <>
struct StorageTraits<float> {
  using R = float;
  static constexpr bool kNeq = false;
  static constexpr bool kPaired = true;
  __device__ static R load(const float* p) { return __ldg(p); }
  __device__ static void store(float* p, R v) { __stcs(p, v); }
  __device__ static float2 load2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
  __device__ static void store2(float* p, float2 v) { __stcs(reinterpret_cast<float2*>(p), v); }
};

__device__ __forceinline__ __half sat_half(float v) {
  // largest finite half is 65504; saturate instead of producing inf
  return __float2half_rn(fminf(fmaxf(v, -65504.f), 65504.f));
}

template <>
struct StorageTraits<__half> {
  using R = float;
  static constexpr bool kNeq = true;
  static constexpr bool kPaired = true;
  __device__ static float load(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static void store(__half* p, float v) { *p = sat_half(v); }
  __device__ static float2 load2(const __half* p) { return __half22float2(__ldg(reinterpret_cast<const __half2*>(p))); }
  __device__ static void store2(__half* p, float2 v) {
    // one saturating conversion of both lanes (round to nearest; values
    // beyond the largest finite half become +-65504, a NaN stays NaN):
    // the same codes as converting and clamping, in one instruction
    unsigned r;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(v.y), "f"(v.x));
    *reinterpret_cast<unsigned*>(p) = r;
  }
};

template <>
struct StorageTraits<__nv_bfloat16> {
  using R = float;
  static constexpr bool kNeq = true;
  static constexpr bool kPaired = true;
  __device__ static float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ static void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ static float2 load2(const __nv_bfloat16* p) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  __device__ static void store2(__nv_bfloat16* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
  }
};

// Element offset of node `cell` (x + 8 y + 64 z) inside a row.
template <typename T>
__host__ __device__ __forceinline__ int node_offset(int cell) {
  if constexpr (StorageTraits<T>::kPaired)
    return 2 * (cell & 255) + (cell >> 8);
  else
    return cell;
}

// Load the moments of node `cell` of block `blk`.
template <typename T>
__device__ __forceinline__ Mom<typename StorageTraits<T>::R> load_node(const T* base, int64_t blk, int cell,
                                                                       const Scales* sc) {
  using Tr = StorageTraits<T>;
  using R = typename Tr::R;
  const T* p = base + blk * (kRows * kCells) + node_offset<T>(cell);
  R v[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) v[r] = Tr::load(p + r * kCells);
  Mom<R> m;
  if constexpr (Tr::kNeq) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) v[r] *= sc->dec[r];
    m.drho = v[0];
    m.ux = v[1];
    m.uy = v[2];
    m.uz = v[3];
    m.sxx = v[4] + v[1] * v[1];
    m.syy = v[5] + v[2] * v[2];
    m.szz = v[6] + v[3] * v[3];
    m.sxy = v[7] + v[1] * v[2];
    m.sxz = v[8] + v[1] * v[3];
    m.syz = v[9] + v[2] * v[3];
  } else {
    m.drho = v[0];
    m.ux = v[1];
    m.uy = v[2];
    m.uz = v[3];
    m.sxx = v[4];
    m.syy = v[5];
    m.szz = v[6];
    m.sxy = v[7];
    m.sxz = v[8];
    m.syz = v[9];
  }
  return m;
}

template <typename T>
__device__ __forceinline__ void store_node(T* base, int64_t blk, int cell, const Mom<typename StorageTraits<T>::R>& m,
                                           const Scales* sc) {
  using Tr = StorageTraits<T>;
  using R = typename Tr::R;
  T* p = base + blk * (kRows * kCells) + node_offset<T>(cell);
  R v[kRows];
  v[0] = m.drho;
  v[1] = m.ux;
  v[2] = m.uy;
  v[3] = m.uz;
  if constexpr (Tr::kNeq) {
    v[4] = m.sxx - m.ux * m.ux;
    v[5] = m.syy - m.uy * m.uy;
    v[6] = m.szz - m.uz * m.uz;
    v[7] = m.sxy - m.ux * m.uy;
    v[8] = m.sxz - m.ux * m.uz;
    v[9] = m.syz - m.uy * m.uz;
#pragma unroll
    for (int r = 0; r < kRows; ++r) v[r] *= sc->enc[r];
  } else {
    v[4] = m.sxx;
    v[5] = m.syy;
    v[6] = m.szz;
    v[7] = m.sxy;
    v[8] = m.sxz;
    v[9] = m.syz;
  }
#pragma unroll
  for (int r = 0; r < kRows; ++r) Tr::store(p + r * kCells, v[r]);
}

// Node pair (x, y, z) / (x, y, z + 4) at pair slot p = x + 8 y + 64 z, z < 4,
// of the paired layouts, as packed values (.x = node z, .y = node z + 4).
template <typename T>
__device__ __forceinline__ Mom<V2> load_pair(const T* base, int64_t blk, int p, const Scales* sc) {
  using Tr = StorageTraits<T>;
  static_assert(Tr::kPaired, "pair access needs a paired layout");
  const T* q = base + blk * (kRows * kCells) + 2 * p;
  V2 v[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) v[r] = V2(Tr::load2(q + r * kCells));
  Mom<V2> m;
  if constexpr (Tr::kNeq) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) v[r] = v[r] * V2(sc->dec[r]);
    m.sxx = v[4] + v[1] * v[1];
    m.syy = v[5] + v[2] * v[2];
    m.szz = v[6] + v[3] * v[3];
    m.sxy = v[7] + v[1] * v[2];
    m.sxz = v[8] + v[1] * v[3];
    m.syz = v[9] + v[2] * v[3];
  } else {
    m.sxx = v[4];
    m.syy = v[5];
    m.szz = v[6];
    m.sxy = v[7];
    m.sxz = v[8];
    m.syz = v[9];
  }
  m.drho = v[0];
  m.ux = v[1];
  m.uy = v[2];
  m.uz = v[3];
  return m;
}

template <typename T>
__device__ __forceinline__ void store_pair(T* base, int64_t blk, int p, const Mom<V2>& m, const Scales* sc) {
  using Tr = StorageTraits<T>;
  static_assert(Tr::kPaired, "pair access needs a paired layout");
  T* q = base + blk * (kRows * kCells) + 2 * p;
  V2 v[kRows];
  v[0] = m.drho;
  v[1] = m.ux;
  v[2] = m.uy;
  v[3] = m.uz;
  if constexpr (Tr::kNeq) {
    v[4] = m.sxx - m.ux * m.ux;
    v[5] = m.syy - m.uy * m.uy;
    v[6] = m.szz - m.uz * m.uz;
    v[7] = m.sxy - m.ux * m.uy;
    v[8] = m.sxz - m.ux * m.uz;
    v[9] = m.syz - m.uy * m.uz;
#pragma unroll
    for (int r = 0; r < kRows; ++r) v[r] = v[r] * V2(sc->enc[r]);
  } else {
    v[4] = m.sxx;
    v[5] = m.syy;
    v[6] = m.szz;
    v[7] = m.sxy;
    v[8] = m.sxz;
    v[9] = m.syz;
  }
#pragma unroll
  for (int r = 0; r < kRows; ++r) Tr::store2(q + r * kCells, v[r].v);
}

}  // namespace hlbm
