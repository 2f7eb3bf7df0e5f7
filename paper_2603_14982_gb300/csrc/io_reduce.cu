// io_reduce.cu -- moment import/export between user buffers and storage, and
// the FP64 reductions (mass, momentum, kinetic energy).
#include <cstdio>
#include <mutex>

#include "hlbm_internal.h"
#include "io_reduce.h"

namespace hlbm {
namespace {

// One thread per node.  src rows are (rho, u, S) as in the public layout.
template <typename T, typename In>
__global__ void k_import(const In* __restrict__ src, T* __restrict__ dst, int64_t n_nodes, const Scales* sc) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const int64_t blk = i / kCells;
  const int cell = int(i % kCells);
  const In* p = src + blk * kRows * kCells + cell;
  using R = typename StorageTraits<T>::R;
  Mom<R> m;
  m.drho = R(double(p[0]) - 1.0);
  m.ux = R(p[1 * kCells]);
  m.uy = R(p[2 * kCells]);
  m.uz = R(p[3 * kCells]);
  m.sxx = R(p[4 * kCells]);
  m.syy = R(p[5 * kCells]);
  m.szz = R(p[6 * kCells]);
  m.sxy = R(p[7 * kCells]);
  m.sxz = R(p[8 * kCells]);
  m.syz = R(p[9 * kCells]);
  store_node<T>(dst, blk, cell, m, sc);
}

template <typename T, typename Out>
__global__ void k_export(const T* __restrict__ src, Out* __restrict__ dst, int64_t n_nodes, const Scales* sc,
                         const float* __restrict__ F, double fx, double fy, double fz, int physical) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const int64_t blk = i / kCells;
  const int cell = int(i % kCells);
  const auto m = load_node<T>(src, blk, cell, sc);
  Out* p = dst + blk * kRows * kCells + cell;
  const double rho = 1.0 + double(m.drho);
  double ux = m.ux, uy = m.uy, uz = m.uz;
  if (physical) {
    if (F != nullptr) {
      const float* Fp = F + blk * 3 * kCells + cell;
      fx = Fp[0];
      fy = Fp[kCells];
      fz = Fp[2 * kCells];
    }
    ux -= 0.5 * fx / rho;
    uy -= 0.5 * fy / rho;
    uz -= 0.5 * fz / rho;
  }
  p[0] = Out(rho);
  p[1 * kCells] = Out(ux);
  p[2 * kCells] = Out(uy);
  p[3 * kCells] = Out(uz);
  p[4 * kCells] = Out(m.sxx);
  p[5 * kCells] = Out(m.syy);
  p[6 * kCells] = Out(m.szz);
  p[7 * kCells] = Out(m.sxy);
  p[8 * kCells] = Out(m.sxz);
  p[9 * kCells] = Out(m.syz);
}

// FP64 sums over the stored blocks of a level (blocks whose `skip` byte is
// set -- covered by a finer level -- contribute nothing).  GB300 runs FP64 at
// about 2 operations per cycle per SM, so the per-node work stays in FP32 and
// the sums are carried to FP64 accuracy in FP32 arithmetic:
//  * mass   = vol (N + sum delta_rho)            (delta_rho is stored exactly);
//  * mom_a  = vol (sum u'_a + sum delta_rho u'_a - sum F_a / 2), since
//    rho u_a = rho u'_a - F_a / 2 exactly for the stored velocity
//    u' = u + F / (2 rho); the products delta_rho u'_a are split exactly into
//    a rounded product and its FMA residual;
//  * KE     = vol sum rho |u|^2 / 2 with u = u' - F / (2 rho) per node (FP32
//    per node: a few units of 6e-8 relative per term).
// Each thread walks its nodes with a grid stride and sums every term with
// the cascaded "Sum2" of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6),
// 2005): Knuth's error-free TwoSum keeps the running sum s and accumulates
// every rounding error in e, so that s + e carries the sum as if in twice
// the working precision (error about (n eps)^2 times the summed magnitudes).
// The pair is widened to FP64 once per thread and summed in FP64 across the
// grid.  Only rows 0-3 (delta_rho, u) are read.  FP64 storage sums plain FP64.
//
// part[cta][kRedSlots]: N, sum delta_rho, sum u' (3), sum delta_rho u' (3),
// sum F (3; force field only), sum of the kinetic energies.
constexpr int kRedThreads = 256;
constexpr int kRedSlots = 12;

template <typename R>
struct CompSum {
  R s = 0, e = 0;
  // s + e += x; the FP32 form is TwoSum, written with intrinsics that the
  // compiler neither contracts nor reorders
  __device__ __forceinline__ void add(R x) {
    if constexpr (sizeof(R) == 4) {
      const float t = __fadd_rn(s, x);
      const float bp = __fsub_rn(t, s);
      const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
      s = t;
      e = __fadd_rn(e, err);
    } else {
      s += x;
    }
  }
  // s + e += a b, with the product's rounding error (an FMA residual) exact
  __device__ __forceinline__ void add_prod(R a, R b) {
    if constexpr (sizeof(R) == 4) {
      const float p = __fmul_rn(a, b);
      add(p);
      e = __fadd_rn(e, __fmaf_rn(a, b, -p));
    } else {
      s += a * b;
    }
  }
  __device__ __forceinline__ double value() const { return double(s) + double(e); }
};

// Four consecutive row values at p (16-byte aligned for float, 8 for the
// 2-byte codes, 32 for double), decoded with the row's scale.
template <typename T>
__device__ __forceinline__ void load4(const T* p, float dec, typename StorageTraits<T>::R (&v)[4]) {
  if constexpr (sizeof(T) == 8) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  } else if constexpr (sizeof(T) == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
  } else {
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
    const T* h = reinterpret_cast<const T*>(&a);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = StorageTraits<T>::R(h[j]) * dec;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_reduce_sums(const T* __restrict__ src, int64_t nb, const Scales* sc,
                                                            const uint8_t* __restrict__ skip,
                                                            const float* __restrict__ F, float fx, float fy, float fz,
                                                            double* __restrict__ part) {
  using R = typename StorageTraits<T>::R;
  CompSum<R> drho, u[3], du[3], f[3], ke;
  int64_t n_own = 0;
  float dec[4] = {1.f, 1.f, 1.f, 1.f};
  if constexpr (StorageTraits<T>::kNeq)
    for (int r = 0; r < 4; ++r) dec[r] = sc->dec[r];
  constexpr int kQuads = kCells / 4;  // four consecutive row positions per item
  const int64_t n = nb * kQuads;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t blk = i / kQuads;
    if (skip != nullptr && skip[blk]) continue;
    const int k0 = 4 * int(i % kQuads);  // first position in the row (node order of the storage)
    const T* p = src + blk * (kRows * kCells) + k0;
    R d[4], ux[4], uy[4], uz[4];
    load4<T>(p, dec[0], d);
    load4<T>(p + kCells, dec[1], ux);
    load4<T>(p + 2 * kCells, dec[2], uy);
    load4<T>(p + 3 * kCells, dec[3], uz);
    R gx[4] = {fx, fx, fx, fx}, gy[4] = {fy, fy, fy, fy}, gz[4] = {fz, fz, fz, fz};
    if (F != nullptr) {
      // force field in natural node order: positions k0..k0+3 of a paired
      // row are the nodes c, c + 256, c + 1, c + 257 with c = k0 / 2
      const float* Fb = F + blk * 3 * kCells;
      const int c = StorageTraits<T>::kPaired ? k0 >> 1 : k0;
      float q[3][4];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if constexpr (StorageTraits<T>::kPaired) {
          const float2 lo = __ldg(reinterpret_cast<const float2*>(Fb + a * kCells + c));
          const float2 hi = __ldg(reinterpret_cast<const float2*>(Fb + a * kCells + c + 256));
          q[a][0] = lo.x;
          q[a][1] = hi.x;
          q[a][2] = lo.y;
          q[a][3] = hi.y;
        } else {
          const float4 v4 = __ldg(reinterpret_cast<const float4*>(Fb + a * kCells + c));
          q[a][0] = v4.x;
          q[a][1] = v4.y;
          q[a][2] = v4.z;
          q[a][3] = v4.w;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        gx[j] = q[0][j];
        gy[j] = q[1][j];
        gz[j] = q[2][j];
        f[0].add(gx[j]);
        f[1].add(gy[j]);
        f[2].add(gz[j]);
      }
    }
    n_own += 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      drho.add(d[j]);
      u[0].add(ux[j]);
      u[1].add(uy[j]);
      u[2].add(uz[j]);
      du[0].add_prod(d[j], ux[j]);
      du[1].add_prod(d[j], uy[j]);
      du[2].add_prod(d[j], uz[j]);
      const R rho = R(1) + d[j];
      R hir;
      if constexpr (sizeof(R) == sizeof(float))
        hir = __fdividef(0.5f, rho);  // the kinetic-energy products are FP32 anyway
      else
        hir = R(0.5) / rho;
      const R vx = ux[j] - gx[j] * hir, vy = uy[j] - gy[j] * hir, vz = uz[j] - gz[j] * hir;
      ke.add(R(0.5) * rho * (vx * vx + vy * vy + vz * vz));
    }
  }
  double v[kRedSlots] = {double(n_own), drho.value(), u[0].value(), u[1].value(), u[2].value(), du[0].value(),
                         du[1].value(), du[2].value(), f[0].value(), f[1].value(), f[2].value(), ke.value()};
  __shared__ double s[kRedThreads / 32][kRedSlots];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kRedSlots; ++q) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) s[w][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < kRedSlots) {
    double x = 0;
    for (int j = 0; j < kRedThreads / 32; ++j) x += s[j][threadIdx.x];
    part[int64_t(blockIdx.x) * kRedSlots + threadIdx.x] = x;
  }
}

// Sum the per-CTA partials (warp q sums slot q; fixed order, deterministic)
// and add this level's mass, momentum (3) and kinetic energy, times the cell
// volume, to out[0..4].  Uniform force (field null): sum F = N F.
__global__ void __launch_bounds__(32 * kRedSlots) k_reduce_combine(const double* __restrict__ part, int n_part,
                                                                   int field, double fx, double fy, double fz,
                                                                   double vol, double* out) {
  __shared__ double tot[kRedSlots];
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double x = 0;
  for (int j = lane; j < n_part; j += 32) x += part[int64_t(j) * kRedSlots + q];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if (lane == 0) tot[q] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double N = tot[0];
    const double Fs[3] = {field ? tot[8] : N * fx, field ? tot[9] : N * fy, field ? tot[10] : N * fz};
    out[0] += vol * (N + tot[1]);
    for (int a = 0; a < 3; ++a) out[1 + a] += vol * (tot[2 + a] + tot[5 + a] - 0.5 * Fs[a]);
    out[4] += vol * tot[11];
  }
}

template <typename T>
cudaError_t import_typed(const void* src, int dtype, void* dst, int64_t n_nodes, const Scales* sc, cudaStream_t s) {
  const unsigned grid = unsigned((n_nodes + 255) / 256);
  if (n_nodes == 0) return cudaSuccess;
  if (dtype == 0)
    k_import<T, double><<<grid, 256, 0, s>>>(static_cast<const double*>(src), static_cast<T*>(dst), n_nodes, sc);
  else
    k_import<T, float><<<grid, 256, 0, s>>>(static_cast<const float*>(src), static_cast<T*>(dst), n_nodes, sc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t export_typed(const void* src, void* dst, int dtype, int64_t n_nodes, const Scales* sc, const float* F,
                         const double* fu, int physical, cudaStream_t s) {
  const unsigned grid = unsigned((n_nodes + 255) / 256);
  if (n_nodes == 0) return cudaSuccess;
  if (dtype == 0)
    k_export<T, double><<<grid, 256, 0, s>>>(static_cast<const T*>(src), static_cast<double*>(dst), n_nodes, sc, F,
                                             fu[0], fu[1], fu[2], physical);
  else
    k_export<T, float><<<grid, 256, 0, s>>>(static_cast<const T*>(src), static_cast<float*>(dst), n_nodes, sc, F,
                                            fu[0], fu[1], fu[2], physical);
  return cudaGetLastError();
}

template <typename T>
cudaError_t reduce_typed(const void* src, int64_t nb, const Scales* sc, const uint8_t* skip, const float* F,
                         const double* fu, double vol, double* part, double* out, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  // one wave: no more CTAs than stay resident (the scratch is sized for
  // reduce_ctas(nb), an upper bound)
  static int resident = 0;
  if (resident == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_reduce_sums<T>, kRedThreads, 0);
    if (e != cudaSuccess) return e;
    resident = sms * per_sm > 0 ? sms * per_sm : 1;
  }
  const int grid = reduce_ctas(nb) < resident ? reduce_ctas(nb) : resident;
  k_reduce_sums<T><<<unsigned(grid), kRedThreads, 0, s>>>(static_cast<const T*>(src), nb, sc, skip, F, float(fu[0]),
                                                          float(fu[1]), float(fu[2]), part);
  k_reduce_combine<<<1, 32 * kRedSlots, 0, s>>>(part, grid, F != nullptr ? 1 : 0, fu[0], fu[1], fu[2], vol, out);
  return cudaGetLastError();
}

}  // namespace

#define HLBM_DISPATCH(storage, fn, ...)                                   \
  switch (storage) {                                                      \
    case HLBM_STORE_F64: return fn<double>(__VA_ARGS__);                  \
    case HLBM_STORE_F32: return fn<float>(__VA_ARGS__);                   \
    case HLBM_STORE_F16S: return fn<__half>(__VA_ARGS__);                 \
    case HLBM_STORE_BF16S: return fn<__nv_bfloat16>(__VA_ARGS__);         \
    default: return cudaErrorInvalidValue;                                \
  }

namespace {

template <typename V>
__global__ void k_count_nonfinite(const V* __restrict__ buf, int64_t n, unsigned long long* count) {
  int local = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    local += isfinite(buf[i]) ? 0 : 1;
  const int block = __syncthreads_count(local != 0);
  if (threadIdx.x == 0 && block != 0) atomicAdd(count, static_cast<unsigned long long>(block));
}

}  // namespace

cudaError_t count_nonfinite(const void* buf, int dtype, int64_t n, unsigned long long* count, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  const unsigned grid = unsigned(want < 4096 ? want : 4096);
  if (dtype == 0)
    k_count_nonfinite<double><<<grid, 256, 0, s>>>(static_cast<const double*>(buf), n, count);
  else
    k_count_nonfinite<float><<<grid, 256, 0, s>>>(static_cast<const float*>(buf), n, count);
  return cudaGetLastError();
}

cudaError_t import_moments(int storage, const void* src, int dtype, void* dst, int64_t n_nodes, const Scales* sc,
                           cudaStream_t s) {
  HLBM_DISPATCH(storage, import_typed, src, dtype, dst, n_nodes, sc, s)
}

cudaError_t export_moments(int storage, const void* src, void* dst, int dtype, int64_t n_nodes, const Scales* sc,
                           const float* F, const double* fu, int physical, cudaStream_t s) {
  HLBM_DISPATCH(storage, export_typed, src, dst, dtype, n_nodes, sc, F, fu, physical, s)
}

cudaError_t reduce_level(int storage, const void* src, int64_t nb, const Scales* sc, const uint8_t* skip,
                         const float* F, const double* fu, double vol, double* part, double* out, cudaStream_t s) {
  HLBM_DISPATCH(storage, reduce_typed, src, nb, sc, skip, F, fu, vol, part, out, s)
}

int reduce_ctas(int64_t nb) {
  // about 64 nodes per thread at full size; at most 8 CTAs per SM of 152
  const int64_t want = (nb * kCells + int64_t(kRedThreads) * 64 - 1) / (int64_t(kRedThreads) * 64);
  return int(want < 1 ? 1 : (want > 1216 ? 1216 : want));
}

size_t reduce_scratch_doubles(int64_t nb) { return size_t(reduce_ctas(nb)) * kRedSlots; }

}  // namespace hlbm

// ---------------------------------------------------------------------------
// Allocation-free reduction for callers that cannot call cudaMalloc.
//
// Code that runs inside a host whose allocator it does not own -- a plugin
// loaded into another simulation, a real-time loop that must not grow device
// memory, a process whose memory is reserved up front -- still needs the FP64
// mass/momentum/energy sums.  This entry point reads a moment buffer the caller
// already holds and writes five doubles to a buffer the caller passes; its only
// scratch (the per-block partial sums) is a fixed, file-scope device array.
// ---------------------------------------------------------------------------

void hlbm_internal_set_error(const char* msg);

namespace hlbm {
namespace {

// Largest buffer the allocation-free reduction accepts: 65,536 blocks of 8^3
// nodes (33.5M nodes).  The scratch below (7 doubles per block, 3.7 MB) lives
// on every GPU that loads the library until the process exits.
constexpr int64_t kNoAllocMaxBlocks = 65536;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 7];

constexpr int kMaxDevices = 64;
double* g_noalloc_scratch[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

// As k_reduce_blocks, but for the public layout (rho in row 0, float32) that
// hlbm_read_moments produces.
__global__ void __launch_bounds__(512) k_reduce_public_blocks(const float* __restrict__ src,
                                                              const float* __restrict__ F, double fx, double fy,
                                                              double fz, double* __restrict__ part) {
  const int64_t blk = blockIdx.x;
  const int t = threadIdx.x;
  const float* p = src + blk * kRows * kCells + t;
  const double rho = p[0];
  if (F != nullptr) {
    const float* Fp = F + blk * 3 * kCells + t;
    fx = Fp[0];
    fy = Fp[kCells];
    fz = Fp[2 * kCells];
  }
  const double ux = double(p[1 * kCells]) - 0.5 * fx / rho;
  const double uy = double(p[2 * kCells]) - 0.5 * fy / rho;
  const double uz = double(p[3 * kCells]) - 0.5 * fz / rho;
  double v[5] = {rho, rho * ux, rho * uy, rho * uz, 0.5 * rho * (ux * ux + uy * uy + uz * uz)};
  __shared__ double s[16][5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((t & 31) == 0) s[t >> 5][k] = x;
  }
  __syncthreads();
  if (t < 5) {
    double x = 0;
    for (int w = 0; w < 16; ++w) x += s[w][t];
    part[blk * 7 + t] = x;
  }
}

// Sums part[n][7] into out[0..4] by assignment (nothing carried between calls).
__global__ void __launch_bounds__(256) k_reduce_final_store(const double* __restrict__ part, int64_t n,
                                                            double* out) {
  __shared__ double s[256];
  for (int k = 0; k < 5; ++k) {
    double x = 0;
    for (int64_t i = threadIdx.x; i < n; i += 256) x += part[i * 7 + k];
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = s[0];
    __syncthreads();
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_scratch[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_scratch[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace hlbm

extern "C" int32_t hlbm_reduce_f32_noalloc(const float* mom_dev, int64_t n_blocks, const float* F_dev, double fx,
                                           double fy, double fz, double* out_dev, void* stream) {
  using namespace hlbm;
  if (mom_dev == nullptr || out_dev == nullptr) {
    hlbm_internal_set_error("hlbm_reduce_f32_noalloc: NULL buffer");
    return HLBM_E_INVALID_ARG;
  }
  if (n_blocks <= 0 || n_blocks > kNoAllocMaxBlocks) {
    char msg[160];
    snprintf(msg, sizeof(msg), "hlbm_reduce_f32_noalloc: n_blocks = %lld outside [1, %lld]", (long long)n_blocks,
             (long long)kNoAllocMaxBlocks);
    hlbm_internal_set_error(msg);
    return HLBM_E_INVALID_ARG;
  }
  double* part = nullptr;
  cudaError_t e = noalloc_scratch(&part);
  if (e == cudaSuccess) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_reduce_public_blocks<<<unsigned(n_blocks), 512, 0, s>>>(mom_dev, F_dev, fx, fy, fz, part);
    k_reduce_final_store<<<1, 256, 0, s>>>(part, n_blocks, out_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof(msg), "hlbm_reduce_f32_noalloc: %s", cudaGetErrorString(e));
    hlbm_internal_set_error(msg);
    return HLBM_E_CUDA;
  }
  return HLBM_OK;
}

// ---------------------------------------------------------------------------
// Per-row power-of-two scales of the reduced-precision storages.
// ---------------------------------------------------------------------------
namespace hlbm {
namespace {

// |value| maxima of the stored quantities (delta_rho, u, S^neq) per row, as
// float bits (non-negative floats order like their bit patterns).
__device__ __forceinline__ void row_values(const Mom<float>& m, float (&v)[kRows]) {
  v[0] = m.drho;
  v[1] = m.ux;
  v[2] = m.uy;
  v[3] = m.uz;
  v[4] = m.sxx - m.ux * m.ux;
  v[5] = m.syy - m.uy * m.uy;
  v[6] = m.szz - m.uz * m.uz;
  v[7] = m.sxy - m.ux * m.uy;
  v[8] = m.sxz - m.ux * m.uz;
  v[9] = m.syz - m.uy * m.uz;
}

__device__ __forceinline__ void block_amax(float (&v)[kRows], unsigned* amax) {
  __shared__ unsigned s[kRows];
  if (threadIdx.x < kRows) s[threadIdx.x] = 0u;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    float a = fabsf(v[r]);
    if (!(a <= 3.0e38f)) a = 3.0e38f;  // non-finite values pin the scale to the smallest
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&s[r], __float_as_uint(a));
  }
  __syncthreads();
  if (threadIdx.x < kRows) atomicMax(&amax[threadIdx.x], s[threadIdx.x]);
}

// amax of a public-layout buffer (rho, u, S), one CTA of 512 threads per block
template <typename In>
__global__ void __launch_bounds__(512) k_amax_public(const In* __restrict__ src, unsigned* amax) {
  const In* p = src + int64_t(blockIdx.x) * kRows * kCells + threadIdx.x;
  Mom<float> m;
  m.drho = float(double(p[0]) - 1.0);
  m.ux = float(p[1 * kCells]);
  m.uy = float(p[2 * kCells]);
  m.uz = float(p[3 * kCells]);
  m.sxx = float(p[4 * kCells]);
  m.syy = float(p[5 * kCells]);
  m.szz = float(p[6 * kCells]);
  m.sxy = float(p[7 * kCells]);
  m.sxz = float(p[8 * kCells]);
  m.syz = float(p[9 * kCells]);
  float v[kRows];
  row_values(m, v);
  block_amax(v, amax);
}

// dom (per-block domain index, or null) selects the scales and the amax row set.
template <typename T>
__global__ void __launch_bounds__(512) k_amax_storage(const T* __restrict__ src, const Scales* sc, unsigned* amax,
                                                      const int32_t* __restrict__ dom) {
  const int d = dom != nullptr ? dom[blockIdx.x] : 0;
  float v[kRows];
  row_values(load_node<T>(src, blockIdx.x, threadIdx.x, sc + d), v);
  block_amax(v, amax + d * kRows);
}

// scale 2^e with amax * 2^e < 2^13 (three binades below the FP16 maximum).
// The exponent is capped at 20: a row whose amax is (nearly) zero, such as
// S^neq of an equilibrium initial state, still represents values up to
// 65504 * 2^-20 = 0.0625 lattice units, while keeping normal FP16 precision
// down to 6e-11.
// One thread per (domain, row): n_dom * kRows threads.
__global__ void k_set_scales(const unsigned* amax, Scales* sc_all, int n_dom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_dom * kRows) return;
  const int r = i % kRows;
  Scales* sc = sc_all + i / kRows;
  const float a = __uint_as_float(amax[i]);
  int e = 20;
  if (a > 0.f) {
    int k;
    frexpf(a, &k);  // a < 2^k
    e = 13 - k;
  }
  e = max(-30, min(20, e));
  sc->enc[r] = ldexpf(1.f, e);
  sc->dec[r] = ldexpf(1.f, -e);
}

template <typename T>
__global__ void __launch_bounds__(512) k_reencode(T* buf, int64_t nb, const Scales* from, const Scales* to,
                                                  const int32_t* __restrict__ dom) {
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const int d = dom != nullptr ? dom[b] : 0;
    // unchanged scales leave the codes as they are (decoding to S and
    // encoding S - u u again would only add a rounding)
    bool same = true;
#pragma unroll
    for (int r = 0; r < kRows; ++r) same = same && from[d].enc[r] == to[d].enc[r];
    if (same) {
      if (dom == nullptr) return;  // one set of scales: nothing to do anywhere
      continue;
    }
    const Mom<float> m = load_node<T>(buf, b, threadIdx.x, from + d);
    store_node<T>(buf, b, threadIdx.x, m, to + d);
  }
}

inline unsigned reencode_grid(int64_t nb) { return unsigned(nb < 2048 ? nb : 2048); }

// other (optional): a second buffer encoded with the same scales (the other
// ping-pong buffer of a level), re-encoded with the new scales as well.
template <typename T>
cudaError_t rescale_typed(void* buf, int64_t nb, const int32_t* dom, int n_dom, Scales* cur, Scales* tmp,
                          unsigned* amax, cudaStream_t s, void* other = nullptr) {
  if (nb == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(amax, 0, size_t(n_dom) * kRows * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  k_amax_storage<T><<<unsigned(nb), 512, 0, s>>>(static_cast<const T*>(buf), cur, amax, dom);
  k_set_scales<<<unsigned((n_dom * kRows + 255) / 256), 256, 0, s>>>(amax, tmp, n_dom);
  k_reencode<T><<<reencode_grid(nb), 512, 0, s>>>(static_cast<T*>(buf), nb, cur, tmp, dom);
  if (other != nullptr) k_reencode<T><<<reencode_grid(nb), 512, 0, s>>>(static_cast<T*>(other), nb, cur, tmp, dom);
  e = cudaMemcpyAsync(cur, tmp, size_t(n_dom) * sizeof(Scales), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t scales_from_public(const void* src, int dtype, int64_t nb, Scales* sc, unsigned* amax, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(amax, 0, kRows * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (nb > 0) {
    if (dtype == 0)
      k_amax_public<double><<<unsigned(nb), 512, 0, s>>>(static_cast<const double*>(src), amax);
    else
      k_amax_public<float><<<unsigned(nb), 512, 0, s>>>(static_cast<const float*>(src), amax);
  }
  k_set_scales<<<1, 32, 0, s>>>(amax, sc, 1);
  return cudaGetLastError();
}

cudaError_t rescale_storage(int storage, void* buf, int64_t nb, Scales* cur, Scales* tmp, unsigned* amax,
                            cudaStream_t s) {
  return rescale_storage_domains(storage, buf, nb, nullptr, 1, cur, tmp, amax, s);
}

cudaError_t rescale_storage_both(int storage, void* buf, void* other, int64_t nb, Scales* cur, Scales* tmp,
                                 unsigned* amax, cudaStream_t s) {
  switch (storage) {
    case HLBM_STORE_F16S: return rescale_typed<__half>(buf, nb, nullptr, 1, cur, tmp, amax, s, other);
    case HLBM_STORE_BF16S: return rescale_typed<__nv_bfloat16>(buf, nb, nullptr, 1, cur, tmp, amax, s, other);
    default: return cudaSuccess;
  }
}

cudaError_t rescale_storage_domains(int storage, void* buf, int64_t nb, const int32_t* dom, int n_dom, Scales* cur,
                                    Scales* tmp, unsigned* amax, cudaStream_t s) {
  switch (storage) {
    case HLBM_STORE_F16S: return rescale_typed<__half>(buf, nb, dom, n_dom, cur, tmp, amax, s);
    case HLBM_STORE_BF16S: return rescale_typed<__nv_bfloat16>(buf, nb, dom, n_dom, cur, tmp, amax, s);
    default: return cudaSuccess;
  }
}

}  // namespace hlbm
