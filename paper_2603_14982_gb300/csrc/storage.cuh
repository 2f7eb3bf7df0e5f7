// storage.cuh -- moment storage policies.
//
// A level's moments live block-major as [n_blocks][10][512] in one of:
//   double  (80 B/node), float (40 B/node),
//   half / bf16 with a per-row power-of-two scale (20 B/node).
// Row 0 holds delta_rho = rho - 1 for every policy.  The reduced-precision
// policies hold delta_rho, u and S^neq = S - u u, each times 2^e_r with one
// exponent per row and level (the scale is exact, so decoding is
// value = code * 2^-e_r); all arithmetic is done in float.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "lbm_math.cuh"

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
  __device__ static R load(const double* p) { return __ldg(p); }
  __device__ static void store(double* p, R v) { __stcs(p, v); }
};

template <>
struct StorageTraits<float> {
  using R = float;
  static constexpr bool kNeq = false;
  __device__ static R load(const float* p) { return __ldg(p); }
  __device__ static void store(float* p, R v) { __stcs(p, v); }
};

template <>
struct StorageTraits<__half> {
  using R = float;
  static constexpr bool kNeq = true;
  __device__ static float load(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static void store(__half* p, float v) { *p = __float2half_rn(v); }
};

template <>
struct StorageTraits<__nv_bfloat16> {
  using R = float;
  static constexpr bool kNeq = true;
  __device__ static float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ static void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Load the moments of node `cell` of block `blk`.
template <typename T>
__device__ __forceinline__ Mom<typename StorageTraits<T>::R> load_node(const T* base, int64_t blk, int cell,
                                                                       const Scales* sc) {
  using Tr = StorageTraits<T>;
  using R = typename Tr::R;
  const T* p = base + blk * (kRows * kCells) + cell;
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
  T* p = base + blk * (kRows * kCells) + cell;
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

}  // namespace hlbm
