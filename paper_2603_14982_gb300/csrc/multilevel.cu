// multilevel.cu -- downward/upward transfers of Algorithm 1 and the moment
// initialisation of blocks created by a rebuild (Sec. 5.2, Sec. 6.3).
//
// Each stencil node's moments are read from storage and split into
// (delta rho, u, S^neq = S - u u) in FP32 (one fused multiply-add per S^neq
// entry, rounded once); the weighted sums over the stencil and the temporal
// midpoint are accumulated in FP64 with exact power-of-two weights (the
// weights sum to one, so interpolating delta rho = rho - 1 is interpolating
// rho); the result is rescaled and recombined as S = k S^neq + u u (S^eq
// formed from the interpolated velocity) in FP32.  FP64 work is kept to the
// accumulation: on GB300 the FP64 pipe runs at a small fraction of the FP32
// rate, so the widening and the narrowing conversions run on the integer
// pipes.
#include "fp64_bits.cuh"
#include "hlbm_internal.h"
#include "multilevel.cuh"

namespace hlbm {
namespace {

struct Node64 {
  double drho, ux, uy, uz, s[6];  // drho = rho - 1; s = S^neq (xx, yy, zz, xy, xz, yz)
};

template <typename R>
__device__ __forceinline__ R narrow(double v) {
  if constexpr (sizeof(R) == 8)
    return v;
  else
    return to32(v);
}

template <typename M>
__device__ __forceinline__ Node64 split64(const M& m) {
  Node64 n;
  n.drho = to64(m.drho);
  n.ux = to64(m.ux);
  n.uy = to64(m.uy);
  n.uz = to64(m.uz);
  n.s[0] = to64(mad(-m.ux, m.ux, m.sxx));
  n.s[1] = to64(mad(-m.uy, m.uy, m.syy));
  n.s[2] = to64(mad(-m.uz, m.uz, m.szz));
  n.s[3] = to64(mad(-m.ux, m.uy, m.sxy));
  n.s[4] = to64(mad(-m.ux, m.uz, m.sxz));
  n.s[5] = to64(mad(-m.uy, m.uz, m.syz));
  return n;
}

template <typename T>
__device__ __forceinline__ Node64 load64(const void* base, int64_t blk, int cell, const Scales* sc) {
  return split64(load_node<T>(static_cast<const T*>(base), blk, cell, sc));
}

template <typename T>
__device__ __forceinline__ void store64(void* base, int64_t blk, int cell, const Node64& n, double k,
                                        const Scales* sc) {
  using R = typename StorageTraits<T>::R;
  Mom<R> m;
  const R ux = narrow<R>(n.ux), uy = narrow<R>(n.uy), uz = narrow<R>(n.uz), kk = narrow<R>(k);
  m.drho = narrow<R>(n.drho);
  m.ux = ux;
  m.uy = uy;
  m.uz = uz;
  m.sxx = mad(kk, narrow<R>(n.s[0]), ux * ux);
  m.syy = mad(kk, narrow<R>(n.s[1]), uy * uy);
  m.szz = mad(kk, narrow<R>(n.s[2]), uz * uz);
  m.sxy = mad(kk, narrow<R>(n.s[3]), ux * uy);
  m.sxz = mad(kk, narrow<R>(n.s[4]), ux * uz);
  m.syz = mad(kk, narrow<R>(n.s[5]), uy * uz);
  store_node<T>(static_cast<T*>(base), blk, cell, m, sc);
}

__device__ __forceinline__ void axpy(Node64& acc, double w, const Node64& v) {
  acc.drho += w * v.drho;
  acc.ux += w * v.ux;
  acc.uy += w * v.uy;
  acc.uz += w * v.uz;
#pragma unroll
  for (int r = 0; r < 6; ++r) acc.s[r] += w * v.s[r];
}

__device__ __forceinline__ Node64 zero64() {
  Node64 n;
  n.drho = n.ux = n.uy = n.uz = 0.0;
#pragma unroll
  for (int r = 0; r < 6; ++r) n.s[r] = 0.0;
  return n;
}

// Block index holding level node (x, y, z) (node coordinates of that level), or -1.
__device__ __forceinline__ int64_t lookup(const LevelView& v, int x, int y, int z) {
  const int bx = x >> 3, by = y >> 3, bz = z >> 3;
  if (bx < 0 || by < 0 || bz < 0 || bx >= v.d.nx || by >= v.d.ny || bz >= v.d.nz) return -1;
  if (v.hash.keys != nullptr) return hash_find(v.hash, bx, by, bz);
  return v.slot[(int64_t(bz) * v.d.ny + by) * v.d.nx + bx];
}

__device__ __forceinline__ int cell_of(int x, int y, int z) { return (x & 7) + 8 * (y & 7) + 64 * (z & 7); }

// floor(p/2) and ceil(p/2) on a coarse axis of n nodes: ceil wraps on a
// periodic axis and is clamped to the last node on a wall axis.
__device__ __forceinline__ void pair(int p, int n, int periodic, int& lo, int& hi) {
  lo = p >> 1;
  hi = (p + 1) >> 1;
  if (hi >= n) hi = periodic ? hi - n : n - 1;
}

// The adjoint's undo log: the node's stored values before a transfer
// overwrites them (FP32 storage).
template <typename T>
__device__ __forceinline__ void log_node(const TransferArgs& a, int64_t k, int64_t blk, int cell) {
  if constexpr (sizeof(T) == 4) {
    if (a.undo == nullptr) return;
    const T* p = static_cast<const T*>(a.out) + blk * (kRows * kCells) + node_offset<T>(cell);
#pragma unroll
    for (int r = 0; r < kRows; ++r) a.undo[k * kRows + r] = p[r * kCells];
  }
}

// Stencil table of a downward transfer: per fine node, the distinct coarse
// stencil nodes (an even fine index has one coarse node on that axis, an odd
// one two; ceil wraps on a periodic axis and is clamped on a wall axis), in
// the order x fastest, then y, then z.
__global__ void k_down_stencil(TransferArgs a, int32_t* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n_nodes) return;
  const int32_t v = a.nodes[k];
  const int64_t b = v >> 9;
  const int cell = v & 511;
  const int32_t* c = a.fine.coords + 3 * b;
  const int p[3] = {c[0] * 8 + (cell & 7), c[1] * 8 + ((cell >> 3) & 7), c[2] * 8 + (cell >> 6)};
  const int n[3] = {a.coarse.d.nx * 8, a.coarse.d.ny * 8, a.coarse.d.nz * 8};
  int lo[3], hi[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) pair(p[ax], n[ax], a.periodic[ax], lo[ax], hi[ax]);
  const int nx = hi[0] != lo[0] ? 2 : 1, ny = hi[1] != lo[1] ? 2 : 1, nz = hi[2] != lo[2] ? 2 : 1;
  const int nq = nx * ny * nz;
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    int32_t e = -1;
    if (q < nq) {
      const int qx = q % nx, qy = (q / nx) % ny, qz = q / (nx * ny);
      const int x = qx ? hi[0] : lo[0], y = qy ? hi[1] : lo[1], z = qz ? hi[2] : lo[2];
      const int64_t cb = lookup(a.coarse, x, y, z);
      ok = ok && cb >= 0;
      e = cb >= 0 ? int32_t((cb << 9) | cell_of(x, y, z)) : -2;
    }
    out[q * a.n_nodes + k] = e;
  }
  if (!ok) atomicExch(a.status, 1);
}

template <typename T>
__global__ void k_down(TransferArgs a) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n_nodes) return;
  const int32_t v = a.nodes[k];
  const int64_t b = v >> 9;
  const int cell = v & 511;
  // the stencil from the table (built with the hierarchy): at most
  // 2^(odd coordinates) entries, the same number for the whole warp
  const int nmax = (1 + (cell & 1)) * (1 + ((cell >> 3) & 1)) * (1 + ((cell >> 6) & 1));
  int32_t st[8];
  int nq = 0;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    st[q] = q < nmax ? a.stencil[q * a.n_nodes + k] : -1;
    nq += st[q] >= 0 ? 1 : 0;
    bad = bad || st[q] == -2;
  }
  if (bad) {
    atomicExch(a.status, 1);
    return;
  }
  int64_t cb[8];
  int cc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    cb[q] = st[q] >= 0 ? (st[q] >> 9) : 0;
    cc[q] = st[q] & 511;
  }
  // weight 1/nq = 2^-e (exact in FP64), halved once more when the new
  // state's sums are added to half the kept ones (step 2) or averaged with
  // the old state's
  const int e = (nq >= 2 ? 1 : 0) + (nq >= 4 ? 1 : 0) + (nq >= 8 ? 1 : 0) + (a.avg ? 1 : 0);
  const double wt = e == 0 ? 1.0 : e == 1 ? 0.5 : e == 2 ? 0.25 : e == 3 ? 0.125 : 0.0625;
  Node64 acc = zero64();
  const void* cur = a.use_other ? a.coarse.mom_other : a.coarse.mom;
  // step 2 with the old state's sums kept from step 1: half of them plus half
  // the new state's sums (the midpoint is linear in rho, u and S^neq)
  const bool reuse = a.avg && a.acc_old != nullptr;
  if (reuse) {
    const double* o = a.acc_old + k * 10;
    acc.drho = half64(o[0]);
    acc.ux = half64(o[1]);
    acc.uy = half64(o[2]);
    acc.uz = half64(o[3]);
#pragma unroll
    for (int r = 0; r < 6; ++r) acc.s[r] = half64(o[4 + r]);
    cur = a.coarse.mom;
  }
  if (a.avg && !reuse) {
    // temporal midpoint of the old (other) and new (current) coarse states,
    // taken per field on rho, u and S^neq (no sums kept from step 1)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q >= nq) break;
      axpy(acc, wt, load64<T>(a.coarse.mom_other, cb[q], cc[q], a.coarse.sc));
      axpy(acc, wt, load64<T>(a.coarse.mom, cb[q], cc[q], a.coarse.sc));
    }
  } else {
    // the stencil nodes' moments four at a time (nq is the same for the
    // whole warp: the list is in transfer order), then their sums
    using R = typename StorageTraits<T>::R;
    constexpr int G = 4;
#pragma unroll
    for (int q0 = 0; q0 < 8; q0 += G) {
      if (q0 >= nq) break;
      Mom<R> mv[G];
#pragma unroll
      for (int j = 0; j < G; ++j)
        if (q0 + j < nq) mv[j] = load_node<T>(static_cast<const T*>(cur), cb[q0 + j], cc[q0 + j], a.coarse.sc);
#pragma unroll
      for (int j = 0; j < G; ++j)
        if (q0 + j < nq) axpy(acc, wt, split64(mv[j]));
    }
  }
  if (a.use_other && a.acc_old != nullptr) {  // step 1: keep the old state's sums for step 2
    double* o = a.acc_old + k * 10;
    o[0] = acc.drho;
    o[1] = acc.ux;
    o[2] = acc.uy;
    o[3] = acc.uz;
#pragma unroll
    for (int r = 0; r < 6; ++r) o[4 + r] = acc.s[r];
  }
  log_node<T>(a, k, b, cell);
  store64<T>(a.out, b, cell, acc, a.k, a.out_sc);
}

template <typename T>
__global__ void k_up(TransferArgs a) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n_nodes) return;
  const int32_t v = a.nodes[k];
  const int64_t b = v >> 9;
  const int cell = v & 511;
  const int32_t* c = a.coarse.coords + 3 * b;
  const int x = 2 * (c[0] * 8 + (cell & 7)), y = 2 * (c[1] * 8 + ((cell >> 3) & 7)), z = 2 * (c[2] * 8 + (cell >> 6));
  const int64_t fb = lookup(a.fine, x, y, z);
  if (fb < 0) {
    atomicExch(a.status, 1);
    return;
  }
  const Node64 n = load64<T>(a.fine.mom, fb, cell_of(x, y, z), a.fine.sc);
  log_node<T>(a, k, b, cell);
  store64<T>(a.out, b, cell, n, a.k, a.out_sc);
}

// U_l(i): the stored value at level l, else the upward rule applied to U_{l-1}(2i).
template <typename T>
__device__ bool resolve_up(const OldHierarchy& o, int l, int x, int y, int z, Node64& out) {
  for (int m = 0; m <= l; ++m) {
    const int lev = l - m;
    const int px = x << m, py = y << m, pz = z << m;
    const int64_t b = lookup(o.lv[lev], px, py, pz);
    if (b < 0) continue;
    out = load64<T>(o.lv[lev].mom, b, cell_of(px, py, pz), o.lv[lev].sc);
    for (int k = lev; k < l; ++k)
#pragma unroll
      for (int r = 0; r < 6; ++r) out.s[r] *= o.kup[k];
    return true;
  }
  return false;
}

// D_l(i): U_l(i) if defined, else the downward spatial rule over D_{l+1}.
template <typename T, int DEPTH>
__device__ bool resolve(const OldHierarchy& o, int l, int x, int y, int z, Node64& out) {
  if (resolve_up<T>(o, l, x, y, z, out)) return true;
  if constexpr (DEPTH == 0) {
    return false;
  } else {
    if (l >= o.L - 1) return false;
    const int n[3] = {o.ext[0] >> (l + 1), o.ext[1] >> (l + 1), o.ext[2] >> (l + 1)};
    const int p[3] = {x, y, z};
    int lo[3], hi[3];
    for (int ax = 0; ax < 3; ++ax) pair(p[ax], n[ax], o.periodic[ax], lo[ax], hi[ax]);
    Node64 acc = zero64();
    for (int q = 0; q < 8; ++q) {
      Node64 cnode;
      if (!resolve<T, DEPTH - 1>(o, l + 1, (q & 1) ? hi[0] : lo[0], (q & 2) ? hi[1] : lo[1], (q & 4) ? hi[2] : lo[2],
                                 cnode))
        return false;
      axpy(acc, 0.125, cnode);
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) acc.s[r] *= o.kdown[l];
    out = acc;
    return true;
  }
}

// 2 CTAs of 512 threads per SM (at most 64 registers): the copy of surviving
// nodes is the common path; the recursive resolution of new nodes is rare and
// may spill.
template <typename T>
__global__ void __launch_bounds__(512, 2) k_init_level(OldHierarchy o, int level, const int32_t* __restrict__ coords,
                                                    void* out, const Scales* out_sc, int* status) {
  const int64_t b = blockIdx.x;
  const int cell = threadIdx.x;
  const int x = coords[3 * b] * 8 + (cell & 7), y = coords[3 * b + 1] * 8 + ((cell >> 3) & 7),
            z = coords[3 * b + 2] * 8 + (cell >> 6);
  // a node stored at this level before the rebuild keeps its stored codes
  // (the new level starts from the old level's scales).  The lookup depends on
  // the block only, so a block stored before is copied whole by the CTA as one
  // contiguous chunk of 16-byte words.
  const int64_t ob = lookup(o.lv[level], x, y, z);
  if (ob >= 0) {
    constexpr int kWords = int(kRows * kCells * sizeof(T) / sizeof(uint4));
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const T*>(o.lv[level].mom) + ob * (kRows * kCells));
    uint4* dst = reinterpret_cast<uint4*>(static_cast<T*>(out) + b * (kRows * kCells));
    for (int i = cell; i < kWords; i += 512) dst[i] = src[i];
    return;
  }
  Node64 v;
  if (!resolve<T, kMaxLevels - 1>(o, level, x, y, z, v)) {
    atomicExch(status, 2);
    v = zero64();  // rest state
  }
  store64<T>(out, b, cell, v, 1.0, out_sc);
}

// 64-thread CTAs for the transfers: at 130 to 140 registers a thread (the
// downward transfer), seven fit on an SM where one 256-thread CTA did, and
// the last wave of a small launch is finer grained.
constexpr int kTransferThreads = 64;
inline unsigned blocks_for(int64_t n) { return unsigned((n + kTransferThreads - 1) / kTransferThreads); }

template <typename T>
cudaError_t down_typed(const TransferArgs& a, cudaStream_t s) {
  if (a.n_nodes == 0) return cudaSuccess;
  if (a.stencil == nullptr) return cudaErrorInvalidValue;
  k_down<T><<<blocks_for(a.n_nodes), kTransferThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t up_typed(const TransferArgs& a, cudaStream_t s) {
  if (a.n_nodes == 0) return cudaSuccess;
  k_up<T><<<blocks_for(a.n_nodes), kTransferThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t init_typed(const OldHierarchy& o, int level, const int32_t* coords, int64_t nb, void* out,
                       const Scales* out_sc, int* status, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  k_init_level<T><<<unsigned(nb), 512, 0, s>>>(o, level, coords, out, out_sc, status);
  return cudaGetLastError();
}

__global__ void k_test_narrow(const double* __restrict__ in, float* __restrict__ out, float* __restrict__ hw,
                              int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = to32(in[i]);
  hw[i] = __double2float_rn(in[i]);
}

}  // namespace

cudaError_t test_narrow(const double* in, float* out, float* hw, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_test_narrow<<<unsigned((n + 255) / 256), 256, 0, s>>>(in, out, hw, n);
  return cudaGetLastError();
}

#define HLBM_ML_DISPATCH(storage, fn, ...)                        \
  switch (storage) {                                              \
    case HLBM_STORE_F64: return fn<double>(__VA_ARGS__);          \
    case HLBM_STORE_F32: return fn<float>(__VA_ARGS__);           \
    case HLBM_STORE_F16S: return fn<__half>(__VA_ARGS__);         \
    case HLBM_STORE_BF16S: return fn<__nv_bfloat16>(__VA_ARGS__); \
    default: return cudaErrorNotSupported;                        \
  }

cudaError_t down_stencil(const TransferArgs& a, int32_t* out, cudaStream_t s) {
  if (a.n_nodes == 0) return cudaSuccess;
  k_down_stencil<<<blocks_for(a.n_nodes), kTransferThreads, 0, s>>>(a, out);
  return cudaGetLastError();
}

cudaError_t transfer_down(int storage, const TransferArgs& a, cudaStream_t s) {
  HLBM_ML_DISPATCH(storage, down_typed, a, s)
}

cudaError_t transfer_up(int storage, const TransferArgs& a, cudaStream_t s) {
  HLBM_ML_DISPATCH(storage, up_typed, a, s)
}

cudaError_t init_new_level(int storage, const OldHierarchy& old, int level, const int32_t* coords, int64_t nb,
                           void* out, const Scales* out_sc, int* status, cudaStream_t s) {
  HLBM_ML_DISPATCH(storage, init_typed, old, level, coords, nb, out, out_sc, status, s)
}

}  // namespace hlbm
