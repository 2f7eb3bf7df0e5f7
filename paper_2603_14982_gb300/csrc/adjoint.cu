// adjoint.cu -- reverse-mode step of the single-level stream-collide and the
// checkpointed driver behind hlbm_forward_record / hlbm_adjoint.  The paper
// has no adjoint; the forward it reverses is Sec. 3.1 with the Guo force and
// the mixture relaxation time of Sec. 4.
//
// Per reverse step (lambda = dL/dM of the step's output), FP32 storage:
//   the recomputed forward step has recorded its pre-collision moments p;
//   k_adj_collide (elementwise) applies the transposed collision Jacobian to
//     lambda: lambda_p, and adds dL/dF (FP64 sums);
//   k_adj_push2 (node pairs): every node x forms gbar_i(x) = P_i^T lambda_p(x)
//     and hands it back to its pull source x - c_i through the destination-
//     indexed shared buffer of the forward kernel (bounce-back slots take the
//     node's own value); every source y gathers what it fed, takes the weighted
//     moments that transpose its 17 Hermite coefficients and applies
//     (dA/dM)^T at M(y): lambda of the step's input.
// FP64 storage: one node per thread; k_adj_pull recomputes the pull itself,
// k_adj_push is the same reverse stream on a source-indexed buffer.
// All kernels gather; no atomics, so the result is deterministic.
#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "adjoint_math.cuh"
#include "f2_common.cuh"
#include "hlbm_internal.h"
#include "lattice_state.h"

namespace hlbm {
namespace {

// Kernel parameters in the arithmetic type of the one-node-per-thread
// kernels: the float copies for FP32 math (a double-to-float conversion in
// the kernel would run on the FP64 pipe), the doubles for FP64.
template <typename R>
__device__ __forceinline__ R pick(double d, float f) {
  if constexpr (sizeof(R) == sizeof(float))
    return f;
  else
    return d;
}

constexpr int kExt = 10;
constexpr int kExtCells = 1000;
constexpr int kHaloCells = 488;

__host__ __device__ constexpr int slot_of(int j) { return j < 13 ? j : j - 1; }
template <int J>
__host__ __device__ constexpr int ext_off() {
  return Dir<J>::cx + kExt * (Dir<J>::cy + kExt * Dir<J>::cz);
}
__device__ __forceinline__ int ext_index(int x, int y, int z) { return (x + 1) + kExt * ((y + 1) + kExt * (z + 1)); }

// Halo node t of 488: coordinates (-1 or 8 on the face axis) and face 0..5
// (x-, x+, y-, y+, z-, z+); z faces own the 10x10 planes, y faces the 10x8
// remainder, x faces the 8x8 remainder.
__device__ __forceinline__ void halo_cell(int t, int& hx, int& hy, int& hz, int& face) {
  if (t < 200) {
    const int u = t < 100 ? t : t - 100;
    hz = t < 100 ? -1 : 8;
    hx = u % 10 - 1;
    hy = u / 10 - 1;
    face = t < 100 ? 4 : 5;
  } else if (t < 360) {
    const int u = t < 280 ? t - 200 : t - 280;
    hy = t < 280 ? -1 : 8;
    hx = u % 10 - 1;
    hz = u / 10;
    face = t < 280 ? 2 : 3;
  } else {
    const int u = t < 424 ? t - 360 : t - 424;
    hx = t < 424 ? -1 : 8;
    hy = u % 8;
    hz = u / 8;
    face = t < 424 ? 0 : 1;
  }
}

__device__ __forceinline__ int block_dir(int hx, int hy, int hz) {
  const int dx = hx < 0 ? -1 : (hx > 7 ? 1 : 0);
  const int dy = hy < 0 ? -1 : (hy > 7 ? 1 : 0);
  const int dz = hz < 0 ? -1 : (hz > 7 ? 1 : 0);
  return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}

// Sink writing value J to slot J of ext index e (all J), or only those J whose
// component on axis AX equals SG (AX < 0: all).
template <typename R, int AX, int SG>
struct ExtSink {
  R* f;
  int e;
  R g13;
  template <int J>
  __device__ __forceinline__ void put(R v) {
    if constexpr (J == 13) {
      g13 = v;
    } else {
      constexpr int c = AX == 0 ? Dir<J>::cx : (AX == 1 ? Dir<J>::cy : (AX == 2 ? Dir<J>::cz : SG));
      if constexpr (c == SG) f[slot_of(J) * kExtCells + e] = v;
    }
  }
};

template <typename R, int AX, int SG, typename Emit>
__device__ __forceinline__ void emit_face(int face, Emit&& emit, R* f, int e) {
  (void)face;
  ExtSink<R, AX, SG> s{f, e, R(0)};
  emit(s);
}

// Dispatch a sink for halo face `face` with component sign `inward` (+1: the
// directions entering the block, -1: the directions leaving it).
template <typename R, typename Emit>
__device__ __forceinline__ void emit_halo(int face, bool entering, Emit&& emit, R* f, int e) {
  switch (face * 2 + (entering ? 0 : 1)) {
    case 0: emit_face<R, 0, 1>(face, emit, f, e); break;
    case 1: emit_face<R, 0, -1>(face, emit, f, e); break;
    case 2: emit_face<R, 0, -1>(face, emit, f, e); break;
    case 3: emit_face<R, 0, 1>(face, emit, f, e); break;
    case 4: emit_face<R, 1, 1>(face, emit, f, e); break;
    case 5: emit_face<R, 1, -1>(face, emit, f, e); break;
    case 6: emit_face<R, 1, -1>(face, emit, f, e); break;
    case 7: emit_face<R, 1, 1>(face, emit, f, e); break;
    case 8: emit_face<R, 2, 1>(face, emit, f, e); break;
    case 9: emit_face<R, 2, -1>(face, emit, f, e); break;
    case 10: emit_face<R, 2, -1>(face, emit, f, e); break;
    default: emit_face<R, 2, 1>(face, emit, f, e); break;
  }
}

// Source-indexed pull gather (forward order): g[J] = f[J][e - c_J].
template <typename R, int J>
__device__ __forceinline__ void pull_one(const R* f, int e, R g13, R (&g)[27]) {
  if constexpr (J == 13)
    g[13] = g13;
  else
    g[J] = f[slot_of(J) * kExtCells + e - ext_off<J>()];
}
// Destination-indexed push gather (reverse order): g[J] = f[J][e + c_J].
template <typename R, int J>
__device__ __forceinline__ void push_one(const R* f, int e, R g13, R (&g)[27]) {
  if constexpr (J == 13)
    g[13] = g13;
  else
    g[J] = f[slot_of(J) * kExtCells + e + ext_off<J>()];
}
template <typename R, bool PULL, int... Js>
__device__ __forceinline__ void gather27(const R* f, int e, R g13, R (&g)[27], std::integer_sequence<int, Js...>) {
  if constexpr (PULL)
    (pull_one<R, Js>(f, e, g13, g), ...);
  else
    (push_one<R, Js>(f, e, g13, g), ...);
}

// Bounce-back fill at a wall / solid position w (block-local hx, hy, hz):
// forward (PULL): f[J][w] = f[opp J][w + c_J]  (the node w + c_J pulls its own opposite)
// reverse:        f[J][w] = f[opp J][w - c_J]  (the source w - c_J fed itself)
template <typename R, bool PULL, int J>
__device__ __forceinline__ void mirror_one(R* f, int eh, int hx, int hy, int hz, bool solid_any,
                                           const uint8_t* s_solid) {
  if constexpr (J != 13) {
    constexpr int sg = PULL ? 1 : -1;
    const int x = hx + sg * Dir<J>::cx, y = hy + sg * Dir<J>::cy, z = hz + sg * Dir<J>::cz;
    if ((unsigned)x < 8u && (unsigned)y < 8u && (unsigned)z < 8u) {
      const int ed = eh + sg * ext_off<J>();
      if (!(solid_any && s_solid[ed])) f[slot_of(J) * kExtCells + eh] = f[slot_of(26 - J) * kExtCells + ed];
    }
  }
}
template <typename R, bool PULL, int... Js>
__device__ __forceinline__ void mirror27(R* f, int eh, int hx, int hy, int hz, bool solid_any, const uint8_t* s_solid,
                                         std::integer_sequence<int, Js...>) {
  (mirror_one<R, PULL, Js>(f, eh, hx, hy, hz, solid_any, s_solid), ...);
}

template <typename R>
__device__ __forceinline__ PreMom<R> load_pm(const float* p, int64_t blk, int cell) {
  const float* q = p + blk * (kRows * kCells) + cell;
  PreMom<R> l;
  l.drho = R(q[0]);
  l.jx = R(q[1 * kCells]);
  l.jy = R(q[2 * kCells]);
  l.jz = R(q[3 * kCells]);
  l.pxx = R(q[4 * kCells]);
  l.pyy = R(q[5 * kCells]);
  l.pzz = R(q[6 * kCells]);
  l.pxy = R(q[7 * kCells]);
  l.pxz = R(q[8 * kCells]);
  l.pyz = R(q[9 * kCells]);
  return l;
}

template <typename R>
__device__ __forceinline__ Mom<R> load_lam(const float* p, int64_t blk, int cell) {
  const float* q = p + blk * (kRows * kCells) + cell;
  Mom<R> l;
  l.drho = R(q[0]);
  l.ux = R(q[1 * kCells]);
  l.uy = R(q[2 * kCells]);
  l.uz = R(q[3 * kCells]);
  l.sxx = R(q[4 * kCells]);
  l.syy = R(q[5 * kCells]);
  l.szz = R(q[6 * kCells]);
  l.sxy = R(q[7 * kCells]);
  l.sxz = R(q[8 * kCells]);
  l.syz = R(q[9 * kCells]);
  return l;
}

template <typename R>
__device__ __forceinline__ void store10(float* p, int64_t blk, int cell, R a0, R a1, R a2, R a3, R a4, R a5, R a6, R a7,
                                        R a8, R a9) {
  float* q = p + blk * (kRows * kCells) + cell;
  q[0] = float(a0);
  q[1 * kCells] = float(a1);
  q[2 * kCells] = float(a2);
  q[3 * kCells] = float(a3);
  q[4 * kCells] = float(a4);
  q[5 * kCells] = float(a5);
  q[6 * kCells] = float(a6);
  q[7 * kCells] = float(a7);
  q[8 * kCells] = float(a8);
  q[9 * kCells] = float(a9);
}

// Emits gbar_J for all J of one node's lambda_p to a sink.
template <typename R>
struct GbEmit {
  PreMom<R> l;
  template <typename S>
  __device__ __forceinline__ void run(S& s) const {
    run_seq(s, std::make_integer_sequence<int, 27>{});
  }
  template <typename S, int... Js>
  __device__ __forceinline__ void run_seq(S& s, std::integer_sequence<int, Js...>) const {
    (s.template put<Js>(gbar<Js>(l)), ...);
  }
};

struct AdjArgs {
  const float* lam;       // dL/dM of the step's output [nb][10][512] (node-pair push: copied at solid nodes)
  float* lamp;            // dL/dp of the pre-collision moments [nb][10][512]
  double* dF;             // accumulated dL/dF [nb][3][512]
  float* dFs;             // FP32 dL/dF of the current checkpoint segment, used instead of dF when set
  float* lam_out;         // dL/dM of the step's input [nb][10][512]
  const float* pre_prev;  // fused push: recorded p of the previous step
  float* lamp_out;        // fused push: dL/dp of the previous step
  const float* lam_add;   // added to the push's output at every node, or null
  float* lam_add_clear;   // the same buffer when it is to be left zero after the read, or null
  float* raw_out;         // fused push: the output at pass-through nodes (solid or interface), or null
};

// Shared part: the block's ext buffer filled with the forward pull (PULL) or
// the reverse push; returns after the mirror barrier.
template <typename T, bool PULL>
__device__ __forceinline__ void fill_ext(const StepArgs& a, const AdjArgs& d, int64_t blk, int t, int* s_nbr,
                                         unsigned& s_wall, uint8_t* s_solid, typename StorageTraits<T>::R* fbuf,
                                         typename StorageTraits<T>::R& g13, bool& solid_any) {
  using R = typename StorageTraits<T>::R;
  const T* in = static_cast<const T*>(a.in);
  if (t < 32) {
    const int v = t < 27 ? a.nbr[blk * 27 + t] : 0;
    const unsigned wb = __ballot_sync(0xffffffffu, t < 27 && v == kWall);
    if (t < 27) s_nbr[t] = v;
    if (t == 0) s_wall = wb;
  }
  solid_any = a.bflags != nullptr && (a.bflags[blk] & kBlockSolidNear);
  const int x = t & 7, y = (t >> 3) & 7, z = t >> 6;
  const int e = ext_index(x, y, z);
  int hx = 0, hy = 0, hz = 0, face = 0, eh = 0, hnb = kMissing, hsrc = 0;
  if (t < kHaloCells) {
    halo_cell(t, hx, hy, hz, face);
    eh = ext_index(hx, hy, hz);
    hsrc = (hx & 7) + 8 * (hy & 7) + 64 * (hz & 7);
  }
  __syncthreads();
  if (t < kHaloCells) hnb = s_nbr[block_dir(hx, hy, hz)];
  if (solid_any) {
    s_solid[e] = a.solid[blk * kCells + t];
    if (t < kHaloCells) s_solid[eh] = hnb >= 0 ? a.solid[int64_t(hnb) * kCells + hsrc] : 0;
    __syncthreads();
  }
  const bool own_solid = solid_any && s_solid[e];
  const R kxyz = pick<R>(a.kxyz, a.kxyzf);
  if constexpr (PULL) {
    ExtSink<R, -1, 0> own{fbuf, e, R(0)};
    if (!own_solid) emit_all(make_coef(load_node<T>(in, blk, t, a.scales_in), kxyz), own);
    g13 = own.g13;
    if (t < kHaloCells && hnb >= 0 && !(solid_any && s_solid[eh])) {
      const Coef<R> c = make_coef(load_node<T>(in, hnb, hsrc, a.scales_in), kxyz);
      emit_halo<R>(face, true, [&](auto& s) { emit_all(c, s); }, fbuf, eh);
    }
  } else {
    // gbar of the own node and of the halo nodes whose pull source is inside
    ExtSink<R, -1, 0> own{fbuf, e, R(0)};
    if (!own_solid) GbEmit<R>{load_pm<R>(d.lamp, blk, t)}.run(own);
    g13 = own.g13;
    if (t < kHaloCells && hnb >= 0 && !(solid_any && s_solid[eh])) {
      const GbEmit<R> gb{load_pm<R>(d.lamp, hnb, hsrc)};
      emit_halo<R>(face, false, [&](auto& s) { gb.run(s); }, fbuf, eh);
    }
  }
  __syncthreads();
  if (s_wall != 0u || solid_any) {
    if (own_solid) mirror27<R, PULL>(fbuf, e, x, y, z, solid_any, s_solid, std::make_integer_sequence<int, 27>{});
    if (t < kHaloCells && (hnb == kWall || (hnb >= 0 && solid_any && s_solid[eh])))
      mirror27<R, PULL>(fbuf, eh, hx, hy, hz, solid_any, s_solid, std::make_integer_sequence<int, 27>{});
    __syncthreads();
  }
}

// Reverse step, part 1: lambda_p and dL/dF.
template <typename T>
__global__ void __launch_bounds__(512, 1) k_adj_pull(StepArgs a, AdjArgs d) {
  using R = typename StorageTraits<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* fbuf = reinterpret_cast<R*>(smem_raw);
  __shared__ int s_nbr[27];
  __shared__ unsigned s_wall;
  __shared__ uint8_t s_solid[kExtCells];
  const int64_t blk = blockIdx.x;
  const int t = threadIdx.x;
  R g13;
  bool solid_any;
  fill_ext<T, true>(a, d, blk, t, s_nbr, s_wall, s_solid, fbuf, g13, solid_any);
  const int e = ext_index(t & 7, (t >> 3) & 7, t >> 6);
  const bool frozen = solid_any && s_solid[e];
  if (frozen) {  // a solid node copies its input: no dependence on the pulls or on F
    store10<R>(d.lamp, blk, t, R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0));
    return;
  }
  R g[27];
  gather27<R, true>(fbuf, e, g13, g, std::make_integer_sequence<int, 27>{});
  const PreMom<R> p = project(g);
  R fx, fy, fz;
  if (a.F != nullptr) {
    const float* Fp = a.F + blk * 3 * kCells + t;
    fx = R(Fp[0]);
    fy = R(Fp[kCells]);
    fz = R(Fp[2 * kCells]);
  } else {
    fx = pick<R>(a.fu[0], a.fuf[0]);
    fy = pick<R>(a.fu[1], a.fuf[1]);
    fz = pick<R>(a.fu[2], a.fuf[2]);
  }
  R om = pick<R>(a.om, a.omf);
  if (a.eps != nullptr) om = R(1) / (pick<R>(a.tau, a.tauf) * R(a.eps[blk * kCells + t]));
  PreMom<R> lp;
  R lfx, lfy, lfz;
  collide_vjp(p, fx, fy, fz, om, load_lam<R>(d.lam, blk, t), lp, lfx, lfy, lfz);
  store10<R>(d.lamp, blk, t, lp.drho, lp.jx, lp.jy, lp.jz, lp.pxx, lp.pyy, lp.pzz, lp.pxy, lp.pxz, lp.pyz);
  double* dF = d.dF + blk * 3 * kCells + t;
  dF[0] += double(lfx);
  dF[kCells] += double(lfy);
  dF[2 * kCells] += double(lfz);
}

// Reverse step, part 2: lambda of the step's input moments.
template <typename T>
__global__ void __launch_bounds__(512, 1) k_adj_push(StepArgs a, AdjArgs d) {
  using R = typename StorageTraits<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* fbuf = reinterpret_cast<R*>(smem_raw);
  __shared__ int s_nbr[27];
  __shared__ unsigned s_wall;
  __shared__ uint8_t s_solid[kExtCells];
  const int64_t blk = blockIdx.x;
  const int t = threadIdx.x;
  R g13;
  bool solid_any;
  fill_ext<T, false>(a, d, blk, t, s_nbr, s_wall, s_solid, fbuf, g13, solid_any);
  const int e = ext_index(t & 7, (t >> 3) & 7, t >> 6);
  const bool frozen = solid_any && s_solid[e];
  const Mom<R> lam = load_lam<R>(d.lam, blk, t);
  if (frozen) {  // M'(y) = M(y)
    store10<R>(d.lam_out, blk, t, lam.drho, lam.ux, lam.uy, lam.uz, lam.sxx, lam.syy, lam.szz, lam.sxy, lam.sxz,
               lam.syz);
    return;
  }
  R gb[27];
  gather27<R, false>(fbuf, e, g13, gb, std::make_integer_sequence<int, 27>{});
  const Coef<R> gh = adjoint_moments(gb);
  // the coefficient Jacobian already carries the weights w_i: ghat includes them
  const Mom<R> lm = coef_vjp(load_node<T>(static_cast<const T*>(a.in), blk, t, a.scales_in), gh, pick<R>(a.kxyz, a.kxyzf));
  store10<R>(d.lam_out, blk, t, lm.drho, lm.ux, lm.uy, lm.uz, lm.sxx, lm.syy, lm.szz, lm.sxy, lm.sxz, lm.syz);
}

// ---------------------------------------------------------------- node-pair reverse step
// FP32 storage: the reverse step on node pairs with packed FP32 arithmetic,
// streaming through the same destination-indexed shared buffer as the forward
// kernel (f2_common.cuh).

// Node values of the reverse stream: lambda_p (float32, natural node order)
// and its transposed projection.  A node hands gbar_J back to its pull source
// x - c_J, i.e. along -c_J: the value it emits for direction K is gbar_{26-K},
// and the gather then holds ghat_{26-J} in slot J.  Bounce-back slots take the
// node's own value the same way.
struct LamSource {
  using Node = PreMom<V2>;
  const float* lp;
  __device__ __forceinline__ Node pair(int64_t b, int cell) const {
    const float* q = lp + b * (kRows * kCells) + cell;
    Node n;
    n.drho = V2(q[0], q[256]);
    n.jx = V2(q[kCells], q[kCells + 256]);
    n.jy = V2(q[2 * kCells], q[2 * kCells + 256]);
    n.jz = V2(q[3 * kCells], q[3 * kCells + 256]);
    n.pxx = V2(q[4 * kCells], q[4 * kCells + 256]);
    n.pyy = V2(q[5 * kCells], q[5 * kCells + 256]);
    n.pzz = V2(q[6 * kCells], q[6 * kCells + 256]);
    n.pxy = V2(q[7 * kCells], q[7 * kCells + 256]);
    n.pxz = V2(q[8 * kCells], q[8 * kCells + 256]);
    n.pyz = V2(q[9 * kCells], q[9 * kCells + 256]);
    return n;
  }
  __device__ __forceinline__ Node own(int64_t b, int cell) const { return pair(b, cell); }
  __device__ __forceinline__ Node two(int ba, int ca, int bb, int cb) const {
    float va[kRows], vb[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      va[r] = ba >= 0 ? lp[int64_t(ba) * (kRows * kCells) + r * kCells + ca] : 0.f;
      vb[r] = bb >= 0 ? lp[int64_t(bb) * (kRows * kCells) + r * kCells + cb] : 0.f;
    }
    Node n;
    n.drho = V2(va[0], vb[0]);
    n.jx = V2(va[1], vb[1]);
    n.jy = V2(va[2], vb[2]);
    n.jz = V2(va[3], vb[3]);
    n.pxx = V2(va[4], vb[4]);
    n.pyy = V2(va[5], vb[5]);
    n.pzz = V2(va[6], vb[6]);
    n.pxy = V2(va[7], vb[7]);
    n.pxz = V2(va[8], vb[8]);
    n.pyz = V2(va[9], vb[9]);
    return n;
  }
  __device__ __forceinline__ static Node zero() {
    Node n;
    n.drho = n.jx = n.jy = n.jz = n.pxx = n.pyy = n.pzz = n.pxy = n.pxz = n.pyz = V2(0.f);
    return n;
  }
  // reflection along axis cls: j and Pi components with an odd count of that axis change sign
  __device__ __forceinline__ static void mirror(Node& n, int cls, V2 sg) {
    if (cls == 0) {
      n.jx = n.jx * sg;
      n.pxy = n.pxy * sg;
      n.pxz = n.pxz * sg;
    } else if (cls == 1) {
      n.jy = n.jy * sg;
      n.pxy = n.pxy * sg;
      n.pyz = n.pyz * sg;
    } else {
      n.jz = n.jz * sg;
      n.pxz = n.pxz * sg;
      n.pyz = n.pyz * sg;
    }
  }
  template <typename S, int... Ks>
  __device__ __forceinline__ static void emit_seq(const Node& n, S& s, std::integer_sequence<int, Ks...>) {
    (s.template put<Ks>(gbar<26 - Ks>(n)), ...);
  }
  template <typename S>
  __device__ __forceinline__ void emit(const Node& n, S& s) const {
    emit_seq(n, s, std::make_integer_sequence<int, 27>{});
  }
};

__device__ __forceinline__ void store_pair10(float* p, int64_t blk, int cell, const V2 (&v)[kRows], bool zlo,
                                             bool zhi) {
  float* q = p + blk * (kRows * kCells) + cell;
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    q[r * kCells] = zlo ? 0.f : v[r].v.x;
    q[r * kCells + 256] = zhi ? 0.f : v[r].v.y;
  }
}

// Transposed collision of a node pair (cells c and c + 256 of block blk) from
// its recorded pre-collision moments p and lambda' = dL/dM of the step's
// output: stores lambda_p = (dC/dp)^T lambda' and adds (dC/dF)^T lambda' to
// dFs_all (FP32, the sum over one checkpoint segment) if set, else to dF_all
// (FP64; skipped when both are null).  Frozen halves (fz_lo / fz_hi: solid
// or interface nodes, which copy their input) get lambda_p = 0 and no force
// term.
__device__ __forceinline__ void collide_adj_pair(const StepArgs& a, int64_t blk, int c, const PreMom<V2>& p,
                                                 const Mom<V2>& lo, bool fz_lo, bool fz_hi, float* lamp,
                                                 double* dF_all, float* dFs_all) {
  V2 fx, fy, fz;
  if (a.F != nullptr) {
    const float* Fp = a.F + blk * 3 * kCells + c;
    fx = V2(__ldg(Fp), __ldg(Fp + 256));
    fy = V2(__ldg(Fp + kCells), __ldg(Fp + kCells + 256));
    fz = V2(__ldg(Fp + 2 * kCells), __ldg(Fp + 2 * kCells + 256));
  } else {
    fx = V2(a.fuf[0]);
    fy = V2(a.fuf[1]);
    fz = V2(a.fuf[2]);
  }
  V2 om = V2(a.omf);
  if (a.eps != nullptr)
    om = inv(V2(a.tauf) * V2(__ldg(a.eps + blk * kCells + c), __ldg(a.eps + blk * kCells + c + 256)));
  PreMom<V2> lp;
  V2 lfx, lfy, lfz;
  collide_vjp(p, fx, fy, fz, om, lo, lp, lfx, lfy, lfz);
  const V2 out[kRows] = {lp.drho, lp.jx, lp.jy, lp.jz, lp.pxx, lp.pyy, lp.pzz, lp.pxy, lp.pxz, lp.pyz};
  store_pair10(lamp, blk, c, out, fz_lo, fz_hi);
  if (dFs_all != nullptr) {
    float* dF = dFs_all + blk * 3 * kCells + c;
    if (!fz_lo) {
      dF[0] += lfx.v.x;
      dF[kCells] += lfy.v.x;
      dF[2 * kCells] += lfz.v.x;
    }
    if (!fz_hi) {
      dF[256] += lfx.v.y;
      dF[kCells + 256] += lfy.v.y;
      dF[2 * kCells + 256] += lfz.v.y;
    }
    return;
  }
  if (dF_all == nullptr) return;
  double* dF = dF_all + blk * 3 * kCells + c;
  if (!fz_lo) {
    dF[0] += double(lfx.v.x);
    dF[kCells] += double(lfy.v.x);
    dF[2 * kCells] += double(lfz.v.x);
  }
  if (!fz_hi) {
    dF[256] += double(lfx.v.y);
    dF[kCells + 256] += double(lfy.v.y);
    dF[2 * kCells + 256] += double(lfz.v.y);
  }
}

__device__ __forceinline__ Mom<V2> as_mom(const PreMom<V2>& q) {
  Mom<V2> m;
  m.drho = q.drho;
  m.ux = q.jx;
  m.uy = q.jy;
  m.uz = q.jz;
  m.sxx = q.pxx;
  m.syy = q.pyy;
  m.szz = q.pzz;
  m.sxy = q.pxy;
  m.sxz = q.pxz;
  m.syz = q.pyz;
  return m;
}

// Reverse step, part 2 (node pairs): gbar streamed back to the pull sources,
// weighted moments transposing the 17 Hermite coefficients, (dA/dM)^T at the
// step's input moments: lambda of the step's input.  Solid nodes keep
// lambda = d.lam (nothing streams into them); interface nodes (a neighbour
// block not stored) copy their input in the forward step, so d.lam passes
// through and adds to what streams back from the nodes that pull from them;
// d.lam_add, if set, is added everywhere.  Solid and interface nodes are the
// pass-through nodes; d.lam is read only there.
// kFuse: instead of storing lambda, go on with part 1 of the previous step at
// the same node (its transposed collision needs only this node's lambda and
// recorded p), writing that step's lambda_p to d.lamp_out (zero at
// pass-through nodes, as part 1 leaves it) and its force term to d.dF; lambda
// itself is kept only at the pass-through nodes, in d.raw_out if set (the
// multi-level adjoint reads it there: the transfers' own nodes are interface
// nodes).  d.raw_out may equal d.lam: each thread reads and writes its own
// pair only.
template <typename T, bool kFuse>
__global__ void __launch_bounds__(f2::kThreads, 2) k_adj_push2(StepArgs a, AdjArgs d) {
  extern __shared__ __align__(16) float2 f2buf[];
  __shared__ unsigned s_miss;
  const int64_t blk = blockIdx.x;
  f2::PairCtx cx = f2::pair_ctx();
  const LamSource src{d.lamp};
  f2::stream_pairs(src, a, blk, f2buf, s_miss, cx);
  const int own = cx.own;
  // the fused epilogue's reads from global memory, issued before the gather
  // and the transposed arithmetic so that their latency overlaps them
  PreMom<V2> pp_early;
  Mom<V2> in_early;
  if constexpr (kFuse) {
    pp_early = LamSource{d.pre_prev}.pair(blk, own);
    in_early = load_pair<T>(static_cast<const T*>(a.in), blk, own, a.scales_in);
  }
  bool fz_lo = false, fz_hi = false;  // solid nodes: M'(y) = M(y)
  if (cx.solid_any) {
    fz_lo = a.solid[blk * kCells + own] != 0;
    fz_hi = a.solid[blk * kCells + own + 256] != 0;
  }
  bool cp_lo = false, cp_hi = false;  // interface nodes
  if (s_miss != 0u) {
    cp_lo = !fz_lo && f2::touches_missing(cx.x, cx.y, cx.z0, s_miss);
    cp_hi = !fz_hi && f2::touches_missing(cx.x, cx.y, cx.z0 + 4, s_miss);
  }
  Mom<V2> lm;
  if (!(fz_lo && fz_hi)) {
    V2 g[27];
    f2::gather_all(reinterpret_cast<const float*>(f2buf) + cx.own_p, cx.g13, g,
                   std::make_integer_sequence<int, 27>{});
    if (cp_lo || cp_hi) {
      // an interface node's slots fed from a block that is not stored receive
      // no push (they hold stale values): nothing streams back from there
      const unsigned mlo = cp_lo ? f2::missing_sources(cx.x, cx.y, cx.z0, s_miss) : 0u;
      const unsigned mhi = cp_hi ? f2::missing_sources(cx.x, cx.y, cx.z0 + 4, s_miss) : 0u;
#pragma unroll
      for (int K = 0; K < 27; ++K) {
        if ((mlo >> K) & 1u) g[K].v.x = 0.f;
        if ((mhi >> K) & 1u) g[K].v.y = 0.f;
      }
    }
    V2 gh_in[27];
#pragma unroll
    for (int j = 0; j < 27; ++j) gh_in[j] = g[26 - j];
    const Coef<V2> gh = adjoint_moments(gh_in);
    if constexpr (kFuse)
      lm = coef_vjp(in_early, gh, V2(a.kxyzf));
    else
      lm = coef_vjp(load_pair<T>(static_cast<const T*>(a.in), blk, own, a.scales_in), gh, V2(a.kxyzf));
  }
  V2 out[kRows] = {lm.drho, lm.ux, lm.uy, lm.uz, lm.sxx, lm.syy, lm.szz, lm.sxy, lm.sxz, lm.syz};
  const bool pt_lo = fz_lo || cp_lo, pt_hi = fz_hi || cp_hi;
  if ((pt_lo || pt_hi) && d.lam != nullptr) {
    const PreMom<V2> q = LamSource{d.lam}.pair(blk, own);
    const V2 lam[kRows] = {q.drho, q.jx, q.jy, q.jz, q.pxx, q.pyy, q.pzz, q.pxy, q.pxz, q.pyz};
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const float lo = fz_lo ? lam[r].v.x : (cp_lo ? out[r].v.x + lam[r].v.x : out[r].v.x);
      const float hi = fz_hi ? lam[r].v.y : (cp_hi ? out[r].v.y + lam[r].v.y : out[r].v.y);
      out[r] = V2(lo, hi);
    }
  }
  if (d.lam_add != nullptr) {
    const PreMom<V2> q = LamSource{d.lam_add}.pair(blk, own);
    const V2 add[kRows] = {q.drho, q.jx, q.jy, q.jz, q.pxx, q.pyy, q.pzz, q.pxy, q.pxz, q.pyz};
#pragma unroll
    for (int r = 0; r < kRows; ++r) out[r] = out[r] + add[r];
    if (d.lam_add_clear != nullptr) {  // this thread is the only reader of its pair
      float* z = d.lam_add_clear + blk * (kRows * kCells) + own;
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        z[r * kCells] = 0.f;
        z[r * kCells + 256] = 0.f;
      }
    }
  }
  if constexpr (kFuse) {
    if (d.raw_out != nullptr && (pt_lo || pt_hi)) {
      float* q = d.raw_out + blk * (kRows * kCells) + own;
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        if (pt_lo) q[r * kCells] = out[r].v.x;
        if (pt_hi) q[r * kCells + 256] = out[r].v.y;
      }
    }
    if (pt_lo && pt_hi) {
      V2 z[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) z[r] = V2(0.f);
      store_pair10(d.lamp_out, blk, own, z, true, true);
      return;
    }
    Mom<V2> lo;
    lo.drho = out[0];
    lo.ux = out[1];
    lo.uy = out[2];
    lo.uz = out[3];
    lo.sxx = out[4];
    lo.syy = out[5];
    lo.szz = out[6];
    lo.sxy = out[7];
    lo.sxz = out[8];
    lo.syz = out[9];
    collide_adj_pair(a, blk, own, pp_early, lo, pt_lo, pt_hi, d.lamp_out, d.dF, d.dFs);
  } else {
    store_pair10(d.lam_out, blk, own, out, false, false);
  }
}

// Reverse step, part 1 from recorded pre-collision moments p (elementwise,
// one thread per node pair: cells t and t + 256).
__global__ void __launch_bounds__(256) k_adj_collide(StepArgs a, const float* __restrict__ pre, AdjArgs d) {
  __shared__ unsigned s_miss;
  const int64_t blk = blockIdx.x;
  const int t = threadIdx.x;
  if (t < 32) {
    const int v = t < 27 ? a.nbr[blk * 27 + t] : 0;
    const unsigned mb = __ballot_sync(0xffffffffu, t < 27 && is_copy_nbr(v));
    if (t == 0) s_miss = mb;
  }
  __syncthreads();
  bool fz_lo = false, fz_hi = false;
  if (a.bflags != nullptr && (a.bflags[blk] & kBlockSolidNear)) {
    fz_lo = a.solid[blk * kCells + t] != 0;
    fz_hi = a.solid[blk * kCells + t + 256] != 0;
  }
  if (s_miss != 0u) {  // interface nodes copy their input: no collision to transpose
    const int x = t & 7, y = (t >> 3) & 7, z = t >> 6;
    fz_lo = fz_lo || f2::touches_missing(x, y, z, s_miss);
    fz_hi = fz_hi || f2::touches_missing(x, y, z + 4, s_miss);
  }
  if (fz_lo && fz_hi) {
    V2 z[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) z[r] = V2(0.f);
    store_pair10(d.lamp, blk, t, z, true, true);
    return;
  }
  collide_adj_pair(a, blk, t, LamSource{pre}.pair(blk, t), as_mom(LamSource{d.lam}.pair(blk, t)), fz_lo, fz_hi,
                   d.lamp, d.dF, d.dFs);
}

StepArgs with_floats(const StepArgs& a_in) {
  StepArgs a = a_in;
  for (int k = 0; k < 3; ++k) a.fuf[k] = float(a.fu[k]);
  a.tauf = float(a.tau);
  a.omf = float(a.om);
  a.kxyzf = float(a.kxyz);
  return a;
}

template <typename T>
cudaError_t launch_adj(const StepArgs& a_in, const AdjArgs& d, cudaStream_t s) {
  StepArgs a = a_in;
  for (int k = 0; k < 3; ++k) a.fuf[k] = float(a.fu[k]);
  a.tauf = float(a.tau);
  a.omf = float(a.om);
  a.kxyzf = float(a.kxyz);
  using R = typename StorageTraits<T>::R;
  const size_t smem = size_t(26) * kExtCells * sizeof(R);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_adj_pull<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_adj_push<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (a.nb == 0) return cudaSuccess;
  k_adj_pull<T><<<unsigned(a.nb), 512, smem, s>>>(a, d);
  k_adj_push<T><<<unsigned(a.nb), 512, smem, s>>>(a, d);
  return cudaGetLastError();
}

__global__ void k_dF_out(const double* __restrict__ dF, float* __restrict__ out, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = float(dF[i]);
}

// The FP64 sum over segments takes one segment's FP32 sum, which restarts at zero.
__global__ void k_dF_flush(double* __restrict__ dF, float* __restrict__ dFs, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    dF[i] += double(dFs[i]);
    dFs[i] = 0.f;
  }
}

}  // namespace

cudaError_t adjoint_step(int storage, const StepArgs& a, const float* lam, float* lamp, double* dF, float* lam_out,
                         cudaStream_t s) {
  AdjArgs d{};
  d.lam = lam;
  d.lamp = lamp;
  d.dF = dF;
  d.lam_out = lam_out;
  switch (storage) {
    case HLBM_STORE_F64: return launch_adj<double>(a, d, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t adjoint_collide(const StepArgs& a_in, const float* pre, const float* lam, float* lamp, double* dF,
                            cudaStream_t s, float* dFs) {
  if (a_in.nb == 0) return cudaSuccess;
  const StepArgs a = with_floats(a_in);
  AdjArgs d{};
  d.lam = lam;
  d.lamp = lamp;
  d.dF = dF;
  d.dFs = dFs;
  k_adj_collide<<<unsigned(a.nb), 256, 0, s>>>(a, pre, d);
  return cudaGetLastError();
}

template <bool kFuse>
cudaError_t launch_push2(const StepArgs& a_in, const AdjArgs& d, cudaStream_t s) {
  const StepArgs a = with_floats(a_in);
  const size_t smem = f2::kBufBytes;
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(k_adj_push2<float, kFuse>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (a.nb == 0) return cudaSuccess;
  k_adj_push2<float, kFuse><<<unsigned(a.nb), f2::kThreads, smem, s>>>(a, d);
  return cudaGetLastError();
}

cudaError_t adjoint_push(const StepArgs& a, const float* lam, const float* lamp, float* lam_out, cudaStream_t s,
                         float* lam_add, bool clear_add) {
  AdjArgs d{};
  d.lam = lam;
  d.lamp = const_cast<float*>(lamp);
  d.lam_out = lam_out;
  d.lam_add = lam_add;
  d.lam_add_clear = clear_add ? lam_add : nullptr;
  return launch_push2<false>(a, d, s);
}

cudaError_t adjoint_push_collide(const StepArgs& a, const float* lamp, const float* pre_prev, float* lamp_out,
                                 double* dF, cudaStream_t s, const float* lam, float* raw_out, float* lam_add,
                                 bool clear_add, float* dFs) {
  AdjArgs d{};
  d.lam = lam;
  d.lamp = const_cast<float*>(lamp);
  d.pre_prev = pre_prev;
  d.lamp_out = lamp_out;
  d.dF = dF;
  d.dFs = dFs;
  d.raw_out = raw_out;
  d.lam_add = lam_add;
  d.lam_add_clear = clear_add ? lam_add : nullptr;
  return launch_push2<true>(a, d, s);
}

cudaError_t adjoint_dF_flush(double* dF, float* dFs, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_dF_flush<<<unsigned((n + 255) / 256), 256, 0, s>>>(dF, dFs, n);
  return cudaGetLastError();
}

cudaError_t adjoint_dF_to_float(const double* dF, float* out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_dF_out<<<unsigned((n + 255) / 256), 256, 0, s>>>(dF, out, n);
  return cudaGetLastError();
}

}  // namespace hlbm
