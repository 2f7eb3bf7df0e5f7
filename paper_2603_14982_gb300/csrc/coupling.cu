// coupling.cu -- the coupled level-0 step of Fig. 4 (Sec. 5.4): streaming
// only (S), the drag exchange (Ex) and the collision (C), with a live drag
// that depends on the streamed fluid velocity.
//
// S is the stream-collide kernel in its streaming-only mode: it writes the
// pre-collision moments p = (delta_rho*, j*, Pi*) of every node.  Ex and C run
// fused, elementwise per node pair: the drag on the fluid is
//   F = kappa * eta * (v_p - u*),  u* = j* / rho*,  eta = 1 - eps,
// (the sediment velocity v_p against the fluid velocity of the streamed
// populations, weighted by the solid fraction of the last particle deposit),
// which is stored as the level-0 force field for the fused steps that follow
// until the next exchange (the MPM side updates every few LBM steps, Sec.
// 5.4), and the node collides with it as in the fused step (Guo forcing,
// mixture tau of Sec. 4).  Interface and solid nodes copy their input.
#include <cuda_runtime.h>

#include <cmath>

#include "f2_common.cuh"
#include "hlbm_internal.h"
#include "lattice_state.h"
#include "lbm_math.cuh"
#include "storage.cuh"
#include "v2.cuh"

namespace hlbm {
namespace {

struct DragArgs {
  const float* pre;  // [nb][10][512] pre-collision moments, natural order
  float* F;          // [nb][3][512] drag written here (natural order)
  float kappa;
  float vp[3];
};

template <typename T>
__global__ void __launch_bounds__(256) k_exchange_collide(StepArgs a, DragArgs d) {
  __shared__ unsigned s_miss;
  const int64_t blk = blockIdx.x;
  const int t = threadIdx.x;  // node pair: cells t and t + 256 (pair slot t of the paired storage)
  if (t < 32) {
    const int v = t < 27 ? a.nbr[blk * 27 + t] : 0;
    const unsigned mb = __ballot_sync(0xffffffffu, t < 27 && is_copy_nbr(v));
    if (t == 0) s_miss = mb;
  }
  __syncthreads();
  const int x = t & 7, y = (t >> 3) & 7, z = t >> 6;
  bool copy_lo = false, copy_hi = false;
  if (a.bflags != nullptr && (a.bflags[blk] & kBlockSolidNear)) {
    copy_lo = a.solid[blk * kCells + t] != 0;
    copy_hi = a.solid[blk * kCells + t + 256] != 0;
  }
  if (s_miss != 0u) {
    copy_lo = copy_lo || f2::touches_missing(x, y, z, s_miss);
    copy_hi = copy_hi || f2::touches_missing(x, y, z + 4, s_miss);
  }
  const T* in = static_cast<const T*>(a.in);
  T* out = static_cast<T*>(a.out);
  float* Fq = d.F + blk * 3 * kCells + t;
  if (copy_lo && copy_hi) {
    store_pair<T>(out, blk, t, load_pair<T>(in, blk, t, a.scales_in), a.scales_out);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Fq[r * kCells] = 0.f;
      Fq[r * kCells + 256] = 0.f;
    }
    return;
  }
  const float* q = d.pre + blk * (kRows * kCells) + t;
  PreMom<V2> p;
  p.drho = V2(q[0], q[256]);
  p.jx = V2(q[kCells], q[kCells + 256]);
  p.jy = V2(q[2 * kCells], q[2 * kCells + 256]);
  p.jz = V2(q[3 * kCells], q[3 * kCells + 256]);
  p.pxx = V2(q[4 * kCells], q[4 * kCells + 256]);
  p.pyy = V2(q[5 * kCells], q[5 * kCells + 256]);
  p.pzz = V2(q[6 * kCells], q[6 * kCells + 256]);
  p.pxy = V2(q[7 * kCells], q[7 * kCells + 256]);
  p.pxz = V2(q[8 * kCells], q[8 * kCells + 256]);
  p.pyz = V2(q[9 * kCells], q[9 * kCells + 256]);
  // Ex: drag from the streamed velocity and the solid fraction
  V2 eps = V2(1.f), om = V2(a.omf);
  if (a.eps != nullptr) {
    eps = V2(__ldg(a.eps + blk * kCells + t), __ldg(a.eps + blk * kCells + t + 256));
    om = inv(V2(a.tauf) * eps);
  }
  const V2 ke = V2(d.kappa) * (V2(1.f) - eps);
  const V2 ir = inv(V2(1.f) + p.drho);
  V2 fx = ke * (V2(d.vp[0]) - p.jx * ir);
  V2 fy = ke * (V2(d.vp[1]) - p.jy * ir);
  V2 fz = ke * (V2(d.vp[2]) - p.jz * ir);
  if (copy_lo || copy_hi) {
    fx = V2(copy_lo ? 0.f : fx.v.x, copy_hi ? 0.f : fx.v.y);
    fy = V2(copy_lo ? 0.f : fy.v.x, copy_hi ? 0.f : fy.v.y);
    fz = V2(copy_lo ? 0.f : fz.v.x, copy_hi ? 0.f : fz.v.y);
  }
  Fq[0] = fx.v.x;
  Fq[256] = fx.v.y;
  Fq[kCells] = fy.v.x;
  Fq[kCells + 256] = fy.v.y;
  Fq[2 * kCells] = fz.v.x;
  Fq[2 * kCells + 256] = fz.v.y;
  // C: the collision of the fused step with this force
  Mom<V2> mo = collide(p, fx, fy, fz, om);
  if (copy_lo || copy_hi) mo = f2::select_halves(mo, load_pair<T>(in, blk, t, a.scales_in), copy_lo, copy_hi);
  store_pair<T>(out, blk, t, mo, a.scales_out);
}

template <typename T>
cudaError_t launch_exchange(const StepArgs& a_in, const DragArgs& d, cudaStream_t s) {
  StepArgs a = a_in;
  a.tauf = float(a.tau);
  a.omf = float(a.om);
  if (a.nb == 0) return cudaSuccess;
  k_exchange_collide<T><<<unsigned(a.nb), 256, 0, s>>>(a, d);
  return cudaGetLastError();
}

}  // namespace

bool exchange_due(const hlbm_lattice* h) { return h->drag_every > 0 && h->l0_steps % h->drag_every == 0; }

int coupled_step(hlbm_lattice* h, const StepArgs& a_in) {
  const int64_t nb = h->lv[0].nb;
  int rc;
  void* pre = nullptr;
  if ((rc = LatticeOps::alloc(h, &pre, size_t(nb) * kRows * kCells * sizeof(float)))) return rc;
  if (h->d_F == nullptr) {  // allocated last: a failed step leaves no unwritten force field behind
    void* p = nullptr;
    if ((rc = LatticeOps::alloc(h, &p, size_t(nb) * 3 * kCells * sizeof(float)))) {
      LatticeOps::release(h, pre);
      return rc;
    }
    h->d_F = static_cast<float*>(p);
  }
  StepArgs a = a_in;
  a.pre_out = static_cast<float*>(pre);
  DragArgs d{};
  d.pre = static_cast<const float*>(pre);
  d.F = h->d_F;
  d.kappa = float(h->drag_kappa);
  for (int k = 0; k < 3; ++k) d.vp[k] = float(h->drag_vp[k]);
  cudaError_t e = launch_stream_only(h->cfg.storage, a, h->stream);
  if (e == cudaSuccess) {
    switch (h->cfg.storage) {
      case HLBM_STORE_F32: e = launch_exchange<float>(a, d, h->stream); break;
      case HLBM_STORE_F16S: e = launch_exchange<__half>(a, d, h->stream); break;
      case HLBM_STORE_BF16S: e = launch_exchange<__nv_bfloat16>(a, d, h->stream); break;
      default: e = cudaErrorInvalidValue;
    }
  }
  LatticeOps::release(h, pre);
  if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "coupled step: %s", cudaGetErrorString(e));
  return HLBM_OK;
}

}  // namespace hlbm

using namespace hlbm;

extern "C" int32_t hlbm_set_drag(hlbm_lattice* h, double kappa, const double vp[3], int32_t exchange_every) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (exchange_every < 0) return fail(h, HLBM_E_INVALID_ARG, "exchange_every must be >= 0");
  if (exchange_every > 0) {
    if (vp == nullptr) return fail(h, HLBM_E_INVALID_ARG, "vp is NULL");
    if (!std::isfinite(kappa) || !std::isfinite(vp[0]) || !std::isfinite(vp[1]) || !std::isfinite(vp[2]))
      return fail(h, HLBM_E_INVALID_ARG, "kappa and vp must be finite");
    if (h->cfg.storage == HLBM_STORE_F64)
      return fail(h, HLBM_E_UNSUPPORTED, "the coupled step needs FP32, FP16- or BF16-scaled storage");
    h->drag_kappa = kappa;
    for (int k = 0; k < 3; ++k) h->drag_vp[k] = vp[k];
  }
  h->drag_every = exchange_every;
  h->l0_steps = 0;
  return HLBM_OK;
}
