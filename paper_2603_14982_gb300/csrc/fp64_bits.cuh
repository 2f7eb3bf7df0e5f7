// fp64_bits.cuh -- exact binary32 <-> binary64 conversions and halving on the
// integer pipes, for the FP64 accumulations of the interface transfers
// (Sec. 5.2, 5.3).  On GB300 the FP64 pipe runs at a small fraction of the
// FP32 rate and also executes the conversion instructions, so the transfers
// keep it for the weighted sums alone.
#pragma once
#include <cuda_runtime.h>

namespace hlbm {
namespace {

// Widening float -> double on the integer pipes.  The conversion is exact:
// for a normal binary32 number the binary64 encoding keeps the sign, rebiases
// the exponent by 1023 - 127 = 896 and appends 29 zero bits to the 23-bit
// fraction, i.e. bits64 = sign | ((bits32 & 0x7fffffff) + (896 << 23)) << 29.
// Zeros map to signed zeros; subnormals, infinities and NaNs (never seen on
// a healthy lattice) take the conversion instruction.  The transfers are
// bound by the FP64 pipe, which the conversion instruction also occupies.
//
// The rare cases call out-of-line functions, so that the common path holds
// no conversion instruction at all: a call that is not taken costs one issue
// slot, whereas a conversion written inline may be predicated rather than
// branched around and then occupy the FP64 pipe on every lane (with inline
// fallbacks the downward transfer issued about as many non-FMA FP64
// instructions as it makes conversions).
__device__ __noinline__ double widen_rare(float v) { return double(v); }
__device__ __noinline__ float narrow_rare(double v) { return __double2float_rn(v); }
__device__ __noinline__ double half_rare(double v) { return 0.5 * v; }

__device__ __forceinline__ double to64(double v) { return v; }
__device__ __forceinline__ double to64(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned a = b & 0x7fffffffu;
  const unsigned long long sign = static_cast<unsigned long long>(b & 0x80000000u) << 32;
  if (a >= 0x7f800000u || (a != 0u && a < 0x00800000u)) return widen_rare(v);
  const unsigned long long mag = a == 0u ? 0ull : (static_cast<unsigned long long>(a) + (896ull << 23)) << 29;
  return __longlong_as_double(static_cast<long long>(sign | mag));
}

// 0.5 v, exact: one off the biased exponent of a normal binary64 number
// whose result stays normal; zeros, the bottom of the normal range,
// subnormals, infinities and NaNs take the multiplication.
__device__ __forceinline__ double half64(double v) {
  const long long bits = __double_as_longlong(v);
  const unsigned ex = unsigned(static_cast<unsigned long long>(bits) >> 52) & 0x7ffu;
  if (ex - 2u > 0x7fcu) return half_rare(v);  // biased exponent outside [2, 2046]
  return __longlong_as_double(bits - (1ll << 52));
}

// Narrowing binary64 -> binary32 with round-to-nearest-even on the integer
// pipes (IEEE 754): for results in the normal binary32 range the 52-bit
// fraction is cut to 23 bits and rounded on the 29 dropped bits, ties to
// even; the carry of a round-up propagates into the exponent (up to
// infinity).  Zeros keep their sign; all other inputs (binary32 subnormal or
// overflow range, infinities, NaNs) take the conversion instruction.
__device__ __forceinline__ float to32(double v) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned hi = unsigned(bits >> 32), lo = unsigned(bits);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 897u > 253u) {  // biased exponent outside [897, 1150]
    if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return narrow_rare(v);
  }
  const unsigned keep = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) ? 1u : 0u;
  return __uint_as_float(((hi & 0x80000000u) | ((ex - 896u) << 23) | keep) + up);
}

}  // namespace
}  // namespace hlbm
