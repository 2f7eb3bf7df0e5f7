// stream_collide.cu -- fused pull-stream + moment-space collision of one level
// with FP64 storage and arithmetic (one node per thread).
//
// One CTA per stored 8^3 block, one thread per node (512 threads).
//  1. every fluid node of the block reconstructs its 27 post-collision
//     populations from its stored moments (Eq. three_order_f) and writes them,
//     source-indexed, into a shared 10^3 halo-extended buffer;
//  2. the 488 halo nodes (read from the 26 neighbour blocks, mostly L2 hits)
//     write only the 9 directions that point into the block;
//  3. wall and solid nodes fill their slots with the bounce-back value of the
//     node they face (half-way bounce-back f_i*(x) = f_opp(i)(M(x)));
//  4. every fluid node pulls its 27 inputs at constant offsets
//     (f_i*(x) = f_i(M(x - c_i)), Eq. lbe_normalized with operator splitting),
//     projects them to moments (Eq. rho_u_stress) and collides (Sec. 3.1,
//     mixture tau of Sec. 4).  Nodes with a neighbour block that is not stored
//     (interface nodes, refilled by the downward/upward transfers of
//     Algorithm 1) and solid nodes copy their input.
#include <utility>

#include "hlbm_internal.h"
#include "lbm_math.cuh"

namespace hlbm {
namespace {

constexpr int kExt = 10;
constexpr int kExtCells = 1000;
constexpr int kHaloCells = 488;

__host__ __device__ constexpr int slot_of(int j) { return j < 13 ? j : j - 1; }

template <int J>
__host__ __device__ constexpr int ext_off() {
  return Dir<J>::cx + kExt * (Dir<J>::cy + kExt * Dir<J>::cz);
}

__device__ __forceinline__ int ext_index(int x, int y, int z) { return (x + 1) + kExt * ((y + 1) + kExt * (z + 1)); }

template <typename R>
struct OwnSink {
  R* f;
  int e;
  R g13;
  template <int J>
  __device__ __forceinline__ void put(R v) {
    if constexpr (J == 13)
      g13 = v;
    else
      f[slot_of(J) * kExtCells + e] = v;
  }
};

// Halo node on the face whose inward direction has component SG along axis AX.
template <typename R, int AX, int SG>
struct HaloSink {
  R* f;
  int e;
  template <int J>
  __device__ __forceinline__ void put(R v) {
    constexpr int c = AX == 0 ? Dir<J>::cx : (AX == 1 ? Dir<J>::cy : Dir<J>::cz);
    if constexpr (c == SG) f[slot_of(J) * kExtCells + e] = v;
  }
};

// Halo node t in [0, 488): (hx, hy, hz) in block-local coordinates (-1 or 8 on
// the face axis) and its face 0..5 = x-, x+, y-, y+, z-, z+.  z faces own the
// full 10x10 planes, y faces the 10x8 remainder, x faces the 8x8 remainder.
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

template <typename R, int J>
__device__ __forceinline__ void gather_one(const R* f, int e, R g13, R (&g)[27]) {
  if constexpr (J == 13)
    g[13] = g13;
  else
    g[J] = f[slot_of(J) * kExtCells + e - ext_off<J>()];
}

template <typename R, int... Js>
__device__ __forceinline__ void gather_all(const R* f, int e, R g13, R (&g)[27], std::integer_sequence<int, Js...>) {
  (gather_one<R, Js>(f, e, g13, g), ...);
}

// Bounce-back fill for a wall or solid node at ext index eh, block-local (hx,hy,hz):
// every fluid block node x = h + c_j pulls direction j from h and must receive
// its own opposite population, which it stored at slot opp(j) of its own index.
template <typename R, int J>
__device__ __forceinline__ void mirror_one(R* f, int eh, int hx, int hy, int hz, bool solid_any,
                                           const uint8_t* s_solid) {
  if constexpr (J != 13) {
    const int x = hx + Dir<J>::cx, y = hy + Dir<J>::cy, z = hz + Dir<J>::cz;
    if ((unsigned)x < 8u && (unsigned)y < 8u && (unsigned)z < 8u) {
      const int ed = eh + ext_off<J>();
      if (!(solid_any && s_solid[ed])) f[slot_of(J) * kExtCells + eh] = f[slot_of(26 - J) * kExtCells + ed];
    }
  }
}

template <typename R, int... Js>
__device__ __forceinline__ void mirror_all(R* f, int eh, int hx, int hy, int hz, bool solid_any,
                                           const uint8_t* s_solid, std::integer_sequence<int, Js...>) {
  (mirror_one<R, Js>(f, eh, hx, hy, hz, solid_any, s_solid), ...);
}

template <typename T>
__global__ void __launch_bounds__(512, 1) k_stream_collide(StepArgs a) {
  using Tr = StorageTraits<T>;
  using R = typename Tr::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* fbuf = reinterpret_cast<R*>(smem_raw);  // [26][1000], rest direction kept in registers
  __shared__ int s_nbr[27];
  __shared__ unsigned s_wall, s_miss;
  __shared__ uint8_t s_solid[kExtCells];

  const int64_t blk = a.blk0 + blockIdx.x;
  const int t = threadIdx.x;
  const T* in = static_cast<const T*>(a.in);
  T* out = static_cast<T*>(a.out);

  if (t < 32) {
    const int v = t < 27 ? a.nbr[blk * 27 + t] : 0;
    const unsigned wb = __ballot_sync(0xffffffffu, t < 27 && v == kWall);
    const unsigned mb = __ballot_sync(0xffffffffu, t < 27 && is_copy_nbr(v));
    if (t < 27) s_nbr[t] = v;
    if (t == 0) {
      s_wall = wb;
      s_miss = mb;
    }
  }
  const bool solid_any = a.bflags != nullptr && (a.bflags[blk] & kBlockSolidNear);
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
  if (solid_any) {  // block-uniform
    s_solid[e] = a.solid[blk * kCells + t];
    if (t < kHaloCells) s_solid[eh] = hnb >= 0 ? a.solid[(int64_t)hnb * kCells + hsrc] : 0;
    __syncthreads();
  }
  const bool own_solid = solid_any && s_solid[e];
  const Scales* sc_in = a.scales_in;
  const R kxyz = R(a.kxyz);

  // 1. own node
  const Mom<R> m = load_node<T>(in, blk, t, sc_in);
  OwnSink<R> own{fbuf, e, R(0)};
  if (!own_solid) emit_all(make_coef(m, kxyz), own);

  // 2. halo node: the 9 inward directions
  if (t < kHaloCells && hnb >= 0 && !(solid_any && s_solid[eh])) {
    const Coef<R> c = make_coef(load_node<T>(in, hnb, hsrc, sc_in), kxyz);
    switch (face) {
      case 0: { HaloSink<R, 0, 1> s{fbuf, eh}; emit_all(c, s); } break;
      case 1: { HaloSink<R, 0, -1> s{fbuf, eh}; emit_all(c, s); } break;
      case 2: { HaloSink<R, 1, 1> s{fbuf, eh}; emit_all(c, s); } break;
      case 3: { HaloSink<R, 1, -1> s{fbuf, eh}; emit_all(c, s); } break;
      case 4: { HaloSink<R, 2, 1> s{fbuf, eh}; emit_all(c, s); } break;
      default: { HaloSink<R, 2, -1> s{fbuf, eh}; emit_all(c, s); } break;
    }
  }
  __syncthreads();

  // 3. half-way bounce-back at walls and solid nodes
  if (s_wall != 0u || solid_any) {  // block-uniform
    if (own_solid) mirror_all<R>(fbuf, e, x, y, z, solid_any, s_solid, std::make_integer_sequence<int, 27>{});
    if (t < kHaloCells && (hnb == kWall || (hnb >= 0 && solid_any && s_solid[eh])))
      mirror_all<R>(fbuf, eh, hx, hy, hz, solid_any, s_solid, std::make_integer_sequence<int, 27>{});
    __syncthreads();
  }

  // 4. gather, project, collide
  bool copy = own_solid;
  if (s_miss != 0u) {
    const unsigned mx = 2u | (x == 0 ? 1u : 0u) | (x == 7 ? 4u : 0u);
    const unsigned my = 2u | (y == 0 ? 1u : 0u) | (y == 7 ? 4u : 0u);
    const unsigned mz = 2u | (z == 0 ? 1u : 0u) | (z == 7 ? 4u : 0u);
    unsigned touched = 0;
#pragma unroll
    for (int iz = 0; iz < 3; ++iz)
#pragma unroll
      for (int iy = 0; iy < 3; ++iy)
        if (((mz >> iz) & 1u) && ((my >> iy) & 1u)) touched |= mx << (3 * iy + 9 * iz);
    copy = copy || (touched & s_miss) != 0u;
  }
  Mom<R> mo = m;
  if (!copy) {
    R g[27];
    gather_all<R>(fbuf, e, own.g13, g, std::make_integer_sequence<int, 27>{});
    const PreMom<R> p = project(g);
    R fx, fy, fz;
    if (a.F != nullptr) {
      const float* Fp = a.F + blk * 3 * kCells + t;
      fx = R(__ldg(Fp));
      fy = R(__ldg(Fp + kCells));
      fz = R(__ldg(Fp + 2 * kCells));
    } else {
      fx = R(a.fu[0]);
      fy = R(a.fu[1]);
      fz = R(a.fu[2]);
    }
    R tau = R(a.tau);
    if (a.eps != nullptr) tau *= R(__ldg(a.eps + blk * kCells + t));
    mo = collide(p, fx, fy, fz, R(1) / tau);
  }
  store_node<T>(out, blk, t, mo, a.scales_out);
}

template <typename T>
cudaError_t launch_typed(const StepArgs& a, cudaStream_t s) {
  using R = typename StorageTraits<T>::R;
  const size_t smem = size_t(26) * kExtCells * sizeof(R);
  static bool configured = false;  // per process; the attribute is per function
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(k_stream_collide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    configured = true;
  }
  if (a.nb == 0) return cudaSuccess;
  k_stream_collide<T><<<(unsigned)a.nb, 512, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stream_collide(int storage, const StepArgs& a, cudaStream_t s) {
  switch (storage) {
    case HLBM_STORE_F64: return launch_typed<double>(a, s);
    default: return launch_stream_collide_f2(storage, a, s);
  }
}

}  // namespace hlbm
