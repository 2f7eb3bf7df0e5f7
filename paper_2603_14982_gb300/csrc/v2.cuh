// v2.cuh -- a pair of FP32 values handled with the packed FP32 instructions of
// sm_100-family GPUs (FADD2 / FMUL2 / FFMA2).  The node arithmetic templates of
// lbm_math.cuh instantiated with V2 advance two lattice nodes per thread at
// the instruction cost of one.
#pragma once
#include <cuda_runtime.h>

namespace hlbm {

struct V2 {
  float2 v;
  __device__ __forceinline__ V2() {}
  __device__ __forceinline__ V2(float2 a) : v(a) {}
  __device__ __forceinline__ V2(float lo, float hi) : v(make_float2(lo, hi)) {}
  __device__ __forceinline__ explicit V2(double s) : v(make_float2(float(s), float(s))) {}
  __device__ __forceinline__ explicit V2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ explicit V2(int s) : v(make_float2(float(s), float(s))) {}
};

__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 operator/(V2 a, V2 b) { return V2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ V2& operator*=(V2& a, V2 b) { return a = a * b; }
__device__ __forceinline__ V2 mad(V2 a, V2 b, V2 c) { return V2(__ffma2_rn(a.v, b.v, c.v)); }
// correctly rounded reciprocal of each lane (equal to 1.0f / x)
__device__ __forceinline__ V2 inv(V2 a) { return V2(__frcp_rn(a.v.x), __frcp_rn(a.v.y)); }
__device__ __forceinline__ V2& operator+=(V2& a, V2 b) { return a = a + b; }
__device__ __forceinline__ V2& operator-=(V2& a, V2 b) { return a = a - b; }

}  // namespace hlbm
