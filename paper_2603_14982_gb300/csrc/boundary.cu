// boundary.cu -- open faces of the domain (Sec. 7, the dune and ripple
// scenes): the convective outflow dM/dt + u_n dM/dn = 0 and the logarithmic
// inlet profile u(h) = u0 ln(1 + beta (h - h0)).
//
// The nodes of an open face layer keep their moments in the stream-collide
// step (their neighbour table marks the blocks beyond the face kOpen, so they
// copy like interface nodes).  After every step of a level, k_open_faces
// writes them from the state before the step:
//   outflow  M_b <- M_b - c (M_b - M_i),  c = clamp(u_n(M_i), 0, 1),
//            M_i the node one step inward, u_n its velocity along the
//            outward normal (first-order upwind, Courant number c);
//   inlet    rho of M_i, u = u(h) along the inward normal, S = u u.
// A node on several open faces takes the first of x-, x+, y-, y+, z-, z+.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "hierarchy.cuh"
#include "hlbm_internal.h"
#include "lattice_state.h"
#include "storage.cuh"

namespace hlbm {
namespace {

struct OpenArgs {
  const void* in;
  void* out;
  const int32_t* open;    // [nb + 1]: blocks with an open neighbour, then their count
  const int32_t* nbr;
  const int32_t* coords;  // [nb][3] block coordinates, or null: dense slot order
  GridDims d;             // block grid of the level
  int64_t nb;
  int level;
  int type[6];
  float u0, beta, h0;
  int axis;  // profile coordinate of the inlet
  const Scales* sc;
};

template <typename R>
__device__ __forceinline__ R comp(const Mom<R>& m, int a) {
  return a == 0 ? m.ux : (a == 1 ? m.uy : m.uz);
}

// The blocks with an open neighbour, one warp per block, in any order (each
// block's face update touches only its own nodes).
__global__ void k_open_list(const int32_t* __restrict__ nbr, int64_t nb, int32_t* __restrict__ list) {
  const int64_t blk = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (blk >= nb) return;
  const bool o = lane < 27 && nbr[blk * 27 + lane] == kOpen;
  if (__ballot_sync(0xffffffffu, o) != 0u && lane == 0) list[atomicAdd(&list[nb], 1)] = int32_t(blk);
}

template <typename T>
__device__ __forceinline__ void open_face_block(const OpenArgs& a, int64_t blk);

// One CTA per listed block, a fixed grid walking the list.
template <typename T>
__global__ void __launch_bounds__(512) k_open_faces(OpenArgs a) {
  const int n = a.open[a.nb];
  for (int i = blockIdx.x; i < n; i += gridDim.x) open_face_block<T>(a, a.open[i]);
}

template <typename T>
__device__ __forceinline__ void open_face_block(const OpenArgs& a, int64_t blk) {
  using R = typename StorageTraits<T>::R;
  const int cell = threadIdx.x;
  int c[3];
  if (a.coords != nullptr) {
    c[0] = a.coords[3 * blk];
    c[1] = a.coords[3 * blk + 1];
    c[2] = a.coords[3 * blk + 2];
  } else {
    c[0] = int(blk % a.d.nx);
    c[1] = int((blk / a.d.nx) % a.d.ny);
    c[2] = int(blk / (int64_t(a.d.nx) * a.d.ny));
  }
  const int loc[3] = {cell & 7, (cell >> 3) & 7, cell >> 6};
  const int n[3] = {a.d.nx * 8, a.d.ny * 8, a.d.nz * 8};
  int f = -1;
  for (int k = 0; k < 6 && f < 0; ++k) {
    const int ax = k >> 1, hi = k & 1;
    if (a.type[k] != 0 && c[ax] * 8 + loc[ax] == (hi ? n[ax] - 1 : 0)) f = k;
  }
  if (f < 0) return;
  const int ax = f >> 1, hi = f & 1;
  int li[3] = {loc[0], loc[1], loc[2]};
  li[ax] += hi ? -1 : 1;  // one node inward: local 0 -> 1, 7 -> 6, same block
  const int icell = li[0] + 8 * li[1] + 64 * li[2];
  const T* in = static_cast<const T*>(a.in);
  const Mom<R> mb = load_node<T>(in, blk, cell, a.sc);
  const Mom<R> mi = load_node<T>(in, blk, icell, a.sc);
  Mom<R> m;
  if (a.type[f] == HLBM_FACE_OUTFLOW) {
    const R un = hi ? comp(mi, ax) : -comp(mi, ax);
    const R cr = un < R(0) ? R(0) : (un > R(1) ? R(1) : un);
    auto upd = [&](R b, R i) { return b - cr * (b - i); };
    m.drho = upd(mb.drho, mi.drho);
    m.ux = upd(mb.ux, mi.ux);
    m.uy = upd(mb.uy, mi.uy);
    m.uz = upd(mb.uz, mi.uz);
    m.sxx = upd(mb.sxx, mi.sxx);
    m.syy = upd(mb.syy, mi.syy);
    m.szz = upd(mb.szz, mi.szz);
    m.sxy = upd(mb.sxy, mi.sxy);
    m.sxz = upd(mb.sxz, mi.sxz);
    m.syz = upd(mb.syz, mi.syz);
  } else {
    // profile coordinate in fine-node units (level-l node i sits at i 2^l)
    const float hpos = float((c[a.axis] * 8 + loc[a.axis]) << a.level);
    const float arg = 1.f + a.beta * (hpos - a.h0);
    const R u = arg > 1.f ? R(a.u0 * logf(arg)) : R(0);
    R uv[3] = {R(0), R(0), R(0)};
    uv[ax] = hi ? -u : u;  // along the inward normal
    m.drho = mi.drho;
    m.ux = uv[0];
    m.uy = uv[1];
    m.uz = uv[2];
    m.sxx = uv[0] * uv[0];
    m.syy = uv[1] * uv[1];
    m.szz = uv[2] * uv[2];
    m.sxy = uv[0] * uv[1];
    m.sxz = uv[0] * uv[2];
    m.syz = uv[1] * uv[2];
  }
  store_node<T>(static_cast<T*>(a.out), blk, cell, m, a.sc);
}

}  // namespace

int LatticeOps::open_lists(hlbm_lattice* h) {
  if (h->open_mask() == 0u || !h->have_blocks) return HLBM_OK;
  for (int l = 0; l < h->cfg.num_levels; ++l) {
    LevelData& L = h->lv[l];
    if (L.nb == 0 || L.d_open != nullptr) continue;
    void* p = nullptr;
    int rc = LatticeOps::alloc(h, &p, size_t(L.nb + 1) * sizeof(int32_t));
    if (rc) return rc;
    L.d_open = static_cast<int32_t*>(p);
    cudaError_t e = cudaMemsetAsync(L.d_open + L.nb, 0, sizeof(int32_t), h->stream);
    if (e == cudaSuccess) {
      k_open_list<<<unsigned((L.nb * 32 + 255) / 256), 256, 0, h->stream>>>(L.d_nbr, L.nb, L.d_open);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "open faces: %s", cudaGetErrorString(e));
  }
  return HLBM_OK;
}

int open_faces_step(hlbm_lattice* h, int level, const void* in, void* out) {
  const LevelData& L = h->lv[level];
  if (L.nb == 0 || h->open_mask() == 0u) return HLBM_OK;
  if (L.d_open == nullptr) return fail(h, HLBM_E_BAD_STATE, "open faces: the block list was not made");
  OpenArgs a{};
  a.in = in;
  a.out = out;
  a.open = L.d_open;
  a.nbr = L.d_nbr;
  a.coords = h->device_hierarchy ? L.d_coords : nullptr;
  int dims[3];
  h->block_dims(level, dims);
  a.d = GridDims{dims[0], dims[1], dims[2]};
  a.nb = L.nb;
  a.level = level;
  for (int f = 0; f < 6; ++f) a.type[f] = h->face_type[f];
  a.u0 = float(h->inlet_u0);
  a.beta = float(h->inlet_beta);
  a.h0 = float(h->inlet_h0);
  a.axis = h->inlet_axis;
  a.sc = L.d_scales;
  const unsigned grid = unsigned(L.nb < 1216 ? L.nb : 1216);  // 8 CTAs of 512 per SM on 152 SMs
  switch (h->cfg.storage) {
    case HLBM_STORE_F64: k_open_faces<double><<<grid, 512, 0, h->stream>>>(a); break;
    case HLBM_STORE_F32: k_open_faces<float><<<grid, 512, 0, h->stream>>>(a); break;
    case HLBM_STORE_F16S: k_open_faces<__half><<<grid, 512, 0, h->stream>>>(a); break;
    case HLBM_STORE_BF16S: k_open_faces<__nv_bfloat16><<<grid, 512, 0, h->stream>>>(a); break;
    default: return fail(h, HLBM_E_INVALID_ARG, "unknown storage");
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "open faces: %s", cudaGetErrorString(e));
  return HLBM_OK;
}

}  // namespace hlbm

using namespace hlbm;

extern "C" int32_t hlbm_set_open_faces(hlbm_lattice* h, const int32_t type[6], double u0, double beta, double h0,
                                       int32_t profile_axis) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (type == nullptr) return fail(h, HLBM_E_INVALID_ARG, "type is NULL");
  bool inlet = false;
  for (int f = 0; f < 6; ++f) {
    if (type[f] < HLBM_FACE_CLOSED || type[f] > HLBM_FACE_INLET)
      return fail(h, HLBM_E_INVALID_ARG, "face %d: unknown type %d", f, type[f]);
    if (type[f] != HLBM_FACE_CLOSED && h->cfg.periodic[f >> 1])
      return fail(h, HLBM_E_INVALID_ARG, "face %d: an open face needs a non-periodic axis", f);
    if (type[f] == HLBM_FACE_INLET) {
      inlet = true;
      if (profile_axis == (f >> 1)) return fail(h, HLBM_E_INVALID_ARG, "the profile axis must lie in the inlet face");
    }
  }
  if (inlet && (!std::isfinite(u0) || !std::isfinite(beta) || !std::isfinite(h0) || profile_axis < 0 || profile_axis > 2))
    return fail(h, HLBM_E_INVALID_ARG, "inlet profile: u0, beta, h0 finite and axis 0..2");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  for (int f = 0; f < 6; ++f) h->face_type[f] = type[f];
  h->inlet_u0 = u0;
  h->inlet_beta = beta;
  h->inlet_h0 = h0;
  h->inlet_axis = profile_axis;
  if (!h->have_blocks) return HLBM_OK;
  // rebuild the neighbour tables and bounce masks of the stored levels (the
  // lists of open blocks are made again by the next step)
  for (int l = 0; l < h->cfg.num_levels; ++l) {
    LevelData& L = h->lv[l];
    void* v = L.d_open;
    LatticeOps::release(h, v);
    L.d_open = nullptr;
    if (L.nb == 0) continue;
    if (h->device_hierarchy) {
      int dims[3];
      h->block_dims(l, dims);
      const cudaError_t e = neighbour_table(L.d_coords, L.nb, L.d_slot, GridDims{dims[0], dims[1], dims[2]},
                                            h->cfg.periodic, h->open_mask(), L.d_nbr, h->stream,
                                            BlockHash{L.d_hkeys, L.d_hvals, L.hcap ? L.hcap - 1u : 0u});
      if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "neighbour table: %s", cudaGetErrorString(e));
    } else {
      std::vector<int32_t> slot_to_idx(size_t(L.nb)), nbr;
      for (int64_t s = 0; s < L.nb; ++s) slot_to_idx[size_t(s)] = int32_t(s);
      LatticeOps::build_nbr(h, l, L.coords, slot_to_idx, nbr);
      const cudaError_t e = cudaMemcpyAsync(L.d_nbr, nbr.data(), nbr.size() * sizeof(int32_t),
                                            cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "neighbour table: %s", cudaGetErrorString(e));
    }
    if ((rc = LatticeOps::bounce(h, L))) return rc;
  }
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "open faces: %s", cudaGetErrorString(e));
  return HLBM_OK;
}
