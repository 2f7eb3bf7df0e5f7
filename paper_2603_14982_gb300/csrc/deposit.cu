// deposit.cu -- per-node solid fraction, fluid fraction and drag force of the
// finest level from a particle cloud (the coupling fields F and eps of Sec. 4).
//
// eta(x) = min(eta_max, per_particle * count(x)) with nearest-node counts
// (floor of the position, clamped to the domain), eps = 1 - eta and
// F = (0, -kappa * eta, 0) while the particles move (F = 0 otherwise).  The
// arithmetic is FP64 and rounded once to float32.  Counts are kept as integers
// in the eps buffer and converted in place.
#include <cuda_runtime.h>

#include <cmath>

#include "hierarchy.cuh"
#include "lattice_state.h"

namespace hlbm {
namespace {

__global__ void k_count_particles(const float* __restrict__ pos, int64_t n, int nx, int ny, int nz, int bdx, int bdy,
                                  const int32_t* __restrict__ slot, BlockHash hash, unsigned* cnt,
                                  unsigned long long* outside) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
  if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) {
    atomicAdd(outside, 1ull);
    return;
  }
  const int x = min(max(int(floorf(px)), 0), nx - 1);
  const int y = min(max(int(floorf(py)), 0), ny - 1);
  const int z = min(max(int(floorf(pz)), 0), nz - 1);
  const int64_t s = (int64_t(z >> 3) * bdy + (y >> 3)) * bdx + (x >> 3);
  const int64_t b = hash.keys != nullptr ? hash_find(hash, x >> 3, y >> 3, z >> 3) : (slot != nullptr ? slot[s] : s);
  if (b < 0) {
    atomicAdd(outside, 1ull);
    return;
  }
  atomicAdd(cnt + b * kCells + (x & 7) + 8 * (y & 7) + 64 * (z & 7), 1u);
}

// eps = 1 - eta and the drag F_y = -kappa eta of the first kTableCounts
// particle counts, evaluated on the host with the formula of k_fields; counts
// at or above `sat` take entry `sat` (eta has reached eta_max there).
constexpr int kTableCounts = 64;
struct FieldTable {
  float eps[kTableCounts];
  float fy[kTableCounts];
  int sat;
};

// The same fields from the table: no FP64 work on the device (the FP64 rate
// of GB300 made the formula the kernel's limit), bit-identical results.
__global__ void k_fields_table(float* eps, float* F, int64_t n_nodes, FieldTable t) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const unsigned c = reinterpret_cast<const unsigned*>(eps)[i];
  const int k = c >= unsigned(t.sat) ? t.sat : int(c);
  eps[i] = t.eps[k];
  const int64_t b = i / kCells, j = i % kCells;
  float* Fb = F + b * 3 * kCells + j;
  Fb[0] = 0.f;
  Fb[kCells] = t.fy[k];
  Fb[2 * kCells] = 0.f;
}

__global__ void k_fields(float* eps, float* F, int64_t n_nodes, double kappa, double eta_max, double per_particle,
                         int moving) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const unsigned c = reinterpret_cast<const unsigned*>(eps)[i];
  const double eta = fmin(eta_max, per_particle * double(c));
  eps[i] = float(1.0 - eta);
  const int64_t b = i / kCells, k = i % kCells;
  float* Fb = F + b * 3 * kCells + k;
  Fb[0] = 0.f;
  Fb[kCells] = moving ? float(-kappa * eta) : 0.f;
  Fb[2 * kCells] = 0.f;
}

}  // namespace
}  // namespace hlbm

using namespace hlbm;

extern "C" int32_t hlbm_deposit_particles(hlbm_lattice* h, const float* pos_xyz, int64_t n, int32_t on_device,
                                          double kappa, double eta_max, double per_particle, int32_t moving,
                                          int64_t* outside) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (n < 0 || (n > 0 && pos_xyz == nullptr)) return fail(h, HLBM_E_INVALID_ARG, "bad particle buffer");
  if (!(eta_max >= 0.0 && eta_max < 1.0) || !(per_particle >= 0.0) || !std::isfinite(kappa))
    return fail(h, HLBM_E_INVALID_ARG, "need 0 <= eta_max < 1, per_particle >= 0 and a finite kappa");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "set blocks before depositing particles");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  ProfScope prof_scope(h, kProfDeposit);
  LevelData& L = h->lv[0];
  if (h->device_hierarchy && L.d_slot == nullptr && L.d_hkeys == nullptr)
    return fail(h, HLBM_E_BAD_STATE, "the finest level has no block table");
  const int64_t n_nodes = L.nb * kCells;
  // every buffer is allocated before any is installed in the handle: a failed
  // call leaves no unwritten force or solid-fraction field for the next step
  void *F = nullptr, *eps = nullptr, *cnt = nullptr, *staged = nullptr;
  auto undo = [&](int r) {
    LatticeOps::release(h, F);
    LatticeOps::release(h, eps);
    LatticeOps::release(h, cnt);
    LatticeOps::release(h, staged);
    return r;
  };
  if (h->d_F == nullptr && (rc = LatticeOps::alloc(h, &F, size_t(n_nodes) * 3 * sizeof(float)))) return undo(rc);
  if (h->d_eps == nullptr && (rc = LatticeOps::alloc(h, &eps, size_t(n_nodes) * sizeof(float)))) return undo(rc);
  if (h->d_count == nullptr && (rc = LatticeOps::alloc(h, &cnt, sizeof(unsigned long long)))) return undo(rc);
  if (!on_device && n > 0 && (rc = LatticeOps::alloc(h, &staged, size_t(n) * 3 * sizeof(float)))) return undo(rc);
  if (F) h->d_F = static_cast<float*>(F);
  if (eps) h->d_eps = static_cast<float*>(eps);
  if (cnt) h->d_count = static_cast<unsigned long long*>(cnt);
  const float* d_pos = pos_xyz;
  cudaError_t e = cudaSuccess;
  if (!on_device && n > 0) {
    e = cudaMemcpyAsync(staged, pos_xyz, size_t(n) * 3 * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    d_pos = static_cast<const float*>(staged);
  }
  int dims[3];
  h->block_dims(0, dims);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_count, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_eps, 0, size_t(n_nodes) * sizeof(float), h->stream);
  if (e == cudaSuccess && n > 0) {
    k_count_particles<<<unsigned((n + 255) / 256), 256, 0, h->stream>>>(
        d_pos, n, h->cfg.nx, h->cfg.ny, h->cfg.nz, dims[0], dims[1], h->device_hierarchy ? L.d_slot : nullptr,
        BlockHash{L.d_hkeys, L.d_hvals, L.hcap ? L.hcap - 1u : 0u},
        reinterpret_cast<unsigned*>(h->d_eps), h->d_count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n_nodes > 0) {
    // the count at which eta reaches eta_max, if the table covers it
    int sat = -1;
    for (int c = 0; c < kTableCounts; ++c)
      if (per_particle * double(c) >= eta_max) {
        sat = c;
        break;
      }
    if (sat >= 0) {
      FieldTable t{};
      t.sat = sat;
      for (int c = 0; c <= sat; ++c) {  // the formula of k_fields, in the same FP64 operations
        const double eta = std::fmin(eta_max, per_particle * double(c));
        t.eps[c] = float(1.0 - eta);
        t.fy[c] = moving ? float(-kappa * eta) : 0.f;
      }
      k_fields_table<<<unsigned((n_nodes + 255) / 256), 256, 0, h->stream>>>(h->d_eps, h->d_F, n_nodes, t);
    } else {
      k_fields<<<unsigned((n_nodes + 255) / 256), 256, 0, h->stream>>>(h->d_eps, h->d_F, n_nodes, kappa, eta_max,
                                                                        per_particle, moving ? 1 : 0);
    }
    e = cudaGetLastError();
  }
  unsigned long long out_h = 0;
  if (e == cudaSuccess && outside != nullptr) {
    e = cudaMemcpyAsync(&out_h, h->d_count, sizeof(out_h), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (staged) LatticeOps::release(h, staged);
  if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "particle deposit: %s", cudaGetErrorString(e));
  if (outside) *outside = int64_t(out_h);
  return HLBM_OK;
}
