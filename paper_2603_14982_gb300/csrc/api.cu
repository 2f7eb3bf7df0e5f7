// api.cu -- the C ABI of libhomelbm.so (declared in include/homelbm.h).
#include <cuda_runtime.h>

#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hlbm_internal.h"
#include "io_reduce.h"
#include "lattice_state.h"
#include "multilevel.cuh"

using namespace hlbm;

namespace {
thread_local std::string g_create_error;
}  // namespace

int hlbm::fail(hlbm_lattice* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return code;
}

namespace {

#define HLBM_CUDA(h, call)                                                                      \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail((h), HLBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t storage_bytes(int storage) {
  switch (storage) {
    case HLBM_STORE_F64: return 8;
    case HLBM_STORE_F32: return 4;
    default: return 2;
  }
}

}  // namespace

// ---------------------------------------------------------------- helpers (lattice_state.h)

namespace hlbm {

int LatticeOps::set_device(hlbm_lattice* h) {
  HLBM_CUDA(h, cudaSetDevice(h->cfg.device));
  // Device buffers come from the device's stream-ordered pool.  Freed memory
  // stays cached in the pool (no release threshold), so that the allocations
  // of a hierarchy rebuild neither map new memory nor synchronise the device.
  static std::atomic<bool> pool_ready[64];
  const int dev = h->cfg.device;
  if (dev >= 0 && dev < 64 && !pool_ready[dev].load()) {
    cudaMemPool_t pool;
    HLBM_CUDA(h, cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t threshold = UINT64_MAX;
    HLBM_CUDA(h, cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold));
    pool_ready[dev].store(true);
  }
  return HLBM_OK;
}

// Allocation failure injected for tests of the error paths (hlbm_inject_alloc_failure):
// the number of device allocations still to succeed, or -1.
static std::atomic<int64_t> g_alloc_fail_after{-1};

bool alloc_failure_injected() {
  int64_t left = g_alloc_fail_after.load();
  while (left >= 0 && !g_alloc_fail_after.compare_exchange_weak(left, left - 1)) {
  }
  return left == 0;
}

ProfScope::ProfScope(hlbm_lattice* h, int cls) : h_(h), cls_(cls) {
  if (!h->prof.on) return;
  if (!h->prof.pool.empty()) {
    a_ = h->prof.pool.back();
    h->prof.pool.pop_back();
  } else if (cudaEventCreate(&a_) != cudaSuccess) {
    cudaGetLastError();
    a_ = nullptr;
    return;
  }
  if (cudaEventRecord(a_, h->stream) != cudaSuccess) {
    cudaGetLastError();
    h->prof.pool.push_back(a_);
    a_ = nullptr;
  }
}

ProfScope::~ProfScope() {
  if (a_ == nullptr) return;
  cudaEvent_t b = nullptr;
  if (!h_->prof.pool.empty()) {
    b = h_->prof.pool.back();
    h_->prof.pool.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    h_->prof.pool.push_back(a_);
    return;
  }
  if (cudaEventRecord(b, h_->stream) != cudaSuccess) {
    cudaGetLastError();
    h_->prof.pool.push_back(a_);
    h_->prof.pool.push_back(b);
    return;
  }
  h_->prof.pending.push_back(Profile::Span{cls_, a_, b});
}

int profile_collect(hlbm_lattice* h) {
  if (h->prof.pending.empty()) return HLBM_OK;
  HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  for (const Profile::Span& sp : h->prof.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
      h->prof.ms[sp.cls] += double(ms);
      ++h->prof.count[sp.cls];
    } else {
      cudaGetLastError();
    }
    h->prof.pool.push_back(sp.a);
    h->prof.pool.push_back(sp.b);
  }
  h->prof.pending.clear();
  return HLBM_OK;
}

int LatticeOps::alloc(hlbm_lattice* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return HLBM_OK;
  if (alloc_failure_injected()) return fail(h, HLBM_E_OOM, "allocation of %zu bytes failed (injected)", bytes);
  cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, HLBM_E_OOM, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  return HLBM_OK;
}

void LatticeOps::release(hlbm_lattice* h, void*& p) {
  if (p) cudaFreeAsync(p, h->stream);
  p = nullptr;
}

void LatticeOps::release_tape(hlbm_lattice* h) {
  if (h->tape == nullptr) return;
  for (void*& p : h->tape->bufs) release(h, p);
  delete h->tape;
  h->tape = nullptr;
}

void LatticeOps::free_level(hlbm_lattice* h, LevelData& L) {
  release(h, L.d_mom[0]);
  release(h, L.d_mom[1]);
  void* v = L.d_nbr;
  release(h, v);
  L.d_nbr = nullptr;
  v = L.d_open;
  release(h, v);
  L.d_open = nullptr;
  v = L.d_bflags;
  release(h, v);
  L.d_bflags = nullptr;
  v = L.d_bmask;
  release(h, v);
  L.d_bmask = nullptr;
  v = L.d_solid;
  release(h, v);
  L.d_solid = nullptr;
  v = L.d_skip;
  release(h, v);
  L.d_skip = nullptr;
  for (void** q : {(void**)&L.d_coords, (void**)&L.d_slot, (void**)&L.d_H, (void**)&L.d_stored, (void**)&L.d_down,
                   (void**)&L.d_down_t, (void**)&L.d_down_stc, (void**)&L.d_up, (void**)&L.d_down_acc, (void**)&L.d_list_flags, (void**)&L.d_scales, (void**)&L.d_amax, (void**)&L.d_hkeys, (void**)&L.d_hvals}) {
    release(h, *q);
  }
  L.hcap = 0;
  L.n_down = L.n_up = 0;
  L.nb = 0;
  L.coords.clear();
  L.flags.clear();
  L.host_lists = false;
}

int LatticeOps::host_lists(hlbm_lattice* h, LevelData& L) {
  if (L.host_lists) return HLBM_OK;
  L.coords.resize(size_t(L.nb) * 3);
  L.flags.resize(size_t(L.nb));
  if (L.nb > 0) {
    HLBM_CUDA(h, cudaMemcpyAsync(L.coords.data(), L.d_coords, size_t(L.nb) * 3 * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(h, cudaMemcpyAsync(L.flags.data(), L.d_list_flags, size_t(L.nb), cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  L.host_lists = true;
  return HLBM_OK;
}

static bool reduced(const hlbm_lattice* h) {
  return h->cfg.storage == HLBM_STORE_F16S || h->cfg.storage == HLBM_STORE_BF16S;
}

int LatticeOps::init_scales(hlbm_lattice* h, LevelData& L) {
  if (!reduced(h)) return HLBM_OK;
  int rc;
  void* p;
  if (L.d_scales == nullptr) {
    if ((rc = alloc(h, &p, 2 * sizeof(Scales)))) return rc;
    L.d_scales = static_cast<Scales*>(p);
  }
  if (L.d_amax == nullptr) {
    if ((rc = alloc(h, &p, kRows * sizeof(unsigned)))) return rc;
    L.d_amax = static_cast<unsigned*>(p);
  }
  HLBM_CUDA(h, scales_from_public(nullptr, 1, 0, L.d_scales, L.d_amax, h->stream));
  L.steps_since_rescale = 0;
  return HLBM_OK;
}

int LatticeOps::maybe_rescale(hlbm_lattice* h, LevelData& L, bool force) {
  if (!reduced(h) || L.nb == 0) return HLBM_OK;
  if (!force && ++L.steps_since_rescale < kRescaleEvery) return HLBM_OK;
  L.steps_since_rescale = 0;
  // both buffers share the scales, and the downward transfer reads the
  // coarser level's previous state after its step: a periodic refit
  // re-encodes that buffer too (a forced refit follows a write or a rebuild,
  // after which the other buffer is rewritten before it is read)
  HLBM_CUDA(h, rescale_storage_both(h->cfg.storage, L.d_mom[L.cur], force ? nullptr : L.d_mom[1 - L.cur], L.nb,
                                    L.d_scales, L.d_scales + 1, L.d_amax, h->stream));
  return HLBM_OK;
}

int LatticeOps::bounce(hlbm_lattice* h, LevelData& L) {
  if (L.nb == 0) return HLBM_OK;
  int rc;
  if (L.d_bflags == nullptr) {
    void* p;
    if ((rc = alloc(h, &p, size_t(L.nb)))) return rc;
    L.d_bflags = static_cast<uint8_t*>(p);
    HLBM_CUDA(h, cudaMemsetAsync(L.d_bflags, 0, size_t(L.nb), h->stream));
  }
  if (L.d_bmask == nullptr) {
    void* p;
    if ((rc = alloc(h, &p, size_t(L.nb) * kCells * sizeof(uint32_t)))) return rc;
    L.d_bmask = static_cast<uint32_t*>(p);
  }
  HLBM_CUDA(h, compute_bounce_masks(L.d_nbr, L.d_solid, L.d_bflags, L.d_bmask, L.nb, h->stream));
  return HLBM_OK;
}

// Host-side neighbour table of a block list on the level's block grid.
void LatticeOps::build_nbr(const hlbm_lattice* h, int level, const std::vector<int32_t>& coords,
                           const std::vector<int32_t>& slot_to_idx, std::vector<int32_t>& nbr) {
  int dims[3];
  h->block_dims(level, dims);
  const int64_t nb = int64_t(coords.size() / 3);
  nbr.assign(size_t(nb) * 27, kMissing);
  for (int64_t b = 0; b < nb; ++b) {
    for (int d = 0; d < 27; ++d) {
      const int off[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
      int q[3];
      bool wall = false, open = false;
      for (int a = 0; a < 3; ++a) {
        q[a] = coords[b * 3 + a] + off[a];
        if (q[a] < 0 || q[a] >= dims[a]) {
          if (h->cfg.periodic[a]) {
            q[a] = (q[a] + dims[a]) % dims[a];
          } else {
            wall = true;
            open = open || ((h->open_mask() >> (2 * a + (q[a] < 0 ? 0 : 1))) & 1u) != 0u;
          }
        }
      }
      if (wall) {
        nbr[b * 27 + d] = open ? kOpen : kWall;
        continue;
      }
      const int64_t slot = (int64_t(q[2]) * dims[1] + q[1]) * dims[0] + q[0];
      nbr[b * 27 + d] = slot_to_idx[slot];
    }
  }
}

}  // namespace hlbm

// ---------------------------------------------------------------- ABI

extern "C" {

const char* hlbm_version(void) { return "homelbm-gb300 0.1 (sm_103a)"; }

const char* hlbm_last_error(const hlbm_lattice* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int32_t hlbm_create(const hlbm_config* cfg, hlbm_lattice** out) {
  if (out == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (cfg == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "cfg is NULL");
  if (cfg->block_edge != 8) return fail(nullptr, HLBM_E_INVALID_ARG, "block_edge must be 8 (got %d)", cfg->block_edge);
  if (cfg->num_levels < 1 || cfg->num_levels > 8)
    return fail(nullptr, HLBM_E_INVALID_ARG, "num_levels must be in [1, 8] (got %d)", cfg->num_levels);
  const int64_t unit = int64_t(8) << (cfg->num_levels - 1);
  const int32_t ext[3] = {cfg->nx, cfg->ny, cfg->nz};
  for (int a = 0; a < 3; ++a)
    if (ext[a] <= 0 || ext[a] % unit != 0)
      return fail(nullptr, HLBM_E_INVALID_ARG, "extent %d on axis %d is not a positive multiple of %lld", ext[a], a,
                  (long long)unit);
  if (!(cfg->tau_finest > 0.5) || !std::isfinite(cfg->tau_finest))
    return fail(nullptr, HLBM_E_INVALID_ARG, "tau_finest must be finite and > 1/2");
  if (cfg->storage < HLBM_STORE_F64 || cfg->storage > HLBM_STORE_BF16S)
    return fail(nullptr, HLBM_E_INVALID_ARG, "unknown storage %d", cfg->storage);
  if (cfg->rescale_mode < HLBM_RESCALE_POST || cfg->rescale_mode > HLBM_RESCALE_PAPER)
    return fail(nullptr, HLBM_E_INVALID_ARG, "unknown rescale_mode %d", cfg->rescale_mode);
  if (cfg->num_levels > 4) return fail(nullptr, HLBM_E_UNSUPPORTED, "at most 4 levels are supported");
  hlbm_lattice* h = new (std::nothrow) hlbm_lattice();
  if (h == nullptr) return fail(nullptr, HLBM_E_OOM, "host allocation failed");
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  h->lv.resize(cfg->num_levels);
  double tau = cfg->tau_finest;
  for (int l = 0; l < cfg->num_levels; ++l) {
    h->lv[l].tau = tau;
    tau = tau / 2.0 + 0.25;  // Sec. 5.2 with k = 1
  }
  // Largest |k_up| or |k_down| accepted.  The transfers multiply the S^neq
  // of a node (S - u u, formed from the stored S) by k, so the rounding of the
  // stored S (about 6e-8 of |S| in FP32) grows by |k|; 100 keeps it below the
  // 1e-5 per-step tolerance of the FP32 path.  FP64 storage rounds at 1.1e-16
  // and accepts 1e6.  The post-collision factor 2 (tau_c - 1)/(tau_f - 1)
  // reaches these bounds where a level's tau is close to 1.
  const double kmax = cfg->storage == HLBM_STORE_F64 ? 1e6 : 100.0;
  for (int l = 0; l + 1 < cfg->num_levels; ++l) {
    const double tf = h->lv[l].tau, tc = h->lv[l + 1].tau;
    if (cfg->rescale_mode == HLBM_RESCALE_POST) {
      const double ku = std::fabs(tf - 1.0) > 0.0 ? 2.0 * (tc - 1.0) / (tf - 1.0) : HUGE_VAL;
      if (!(std::fabs(ku) <= kmax && std::fabs(ku) >= 1.0 / kmax)) {
        delete h;
        return fail(nullptr, HLBM_E_INVALID_ARG,
                    "post-collision rescaling between levels %d and %d (tau %g and %g) needs factors within "
                    "[1/%g, %g] in magnitude, got k_up = %g: move tau_finest away from the value that puts a "
                    "level's tau near 1",
                    l, l + 1, tf, tc, kmax, kmax, ku);
      }
      h->kup[l] = ku;
      h->kdown[l] = 1.0 / h->kup[l];
    } else if (cfg->rescale_mode == HLBM_RESCALE_PRE) {
      h->kup[l] = 2.0 * tc / tf;
      h->kdown[l] = 1.0 / h->kup[l];
    } else {
      h->kup[l] = tc / (2.0 * tf);    // Eq. upload_S as printed
      h->kdown[l] = 2.0 * tc / tf;    // Eq. downward_rescale as printed
    }
  }
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    fail(nullptr, HLBM_E_CUDA, "cudaSetDevice(%d): %s", cfg->device, cudaGetErrorString(e));
    delete h;
    return HLBM_E_CUDA;
  }
  *out = h;
  return HLBM_OK;
}

int32_t hlbm_destroy(hlbm_lattice* h) {
  if (h == nullptr) return HLBM_OK;
  cudaSetDevice(h->cfg.device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& L : h->lv) LatticeOps::free_level(h, L);
  LatticeOps::release(h, h->d_stage);
  for (void*& c : h->ckpt) LatticeOps::release(h, c);
  LatticeOps::release_tape(h);
  void* v = h->d_status;
  LatticeOps::release(h, v);
  v = h->d_prev_occ;
  LatticeOps::release(h, v);
  v = h->d_red;
  LatticeOps::release(h, v);
  v = h->d_F;
  LatticeOps::release(h, v);
  v = h->d_eps;
  LatticeOps::release(h, v);
  v = h->d_count;
  LatticeOps::release(h, v);
  if (h->stream) cudaStreamSynchronize(h->stream);  // the frees are ordered on the stream
  for (const Profile::Span& sp : h->prof.pending) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  delete h;
  return HLBM_OK;
}

int32_t hlbm_set_dense(hlbm_lattice* h) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (h->cfg.num_levels != 1) return fail(h, HLBM_E_INVALID_ARG, "hlbm_set_dense needs a single-level lattice");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  LevelData& L = h->lv[0];
  LatticeOps::free_level(h, L);
  h->have_blocks = false;  // until every buffer of the new layout is in place
  int dims[3];
  h->block_dims(0, dims);
  const int64_t nb = int64_t(dims[0]) * dims[1] * dims[2];
  L.coords.resize(size_t(nb) * 3);
  std::vector<int32_t> slot_to_idx(static_cast<size_t>(nb));
  for (int64_t s = 0; s < nb; ++s) {
    L.coords[s * 3 + 0] = int32_t(s % dims[0]);
    L.coords[s * 3 + 1] = int32_t((s / dims[0]) % dims[1]);
    L.coords[s * 3 + 2] = int32_t(s / (int64_t(dims[0]) * dims[1]));
    slot_to_idx[s] = int32_t(s);
  }
  L.flags.assign(size_t(nb), 1);  // leaf
  L.host_lists = true;
  std::vector<int32_t> nbr;
  LatticeOps::build_nbr(h, 0, L.coords, slot_to_idx, nbr);
  L.nb = nb;
  const size_t mom_bytes = size_t(nb) * kRows * kCells * storage_bytes(h->cfg.storage);
  void* p = nullptr;
  if ((rc = LatticeOps::alloc(h, &p, nbr.size() * sizeof(int32_t)))) return rc;
  L.d_nbr = static_cast<int32_t*>(p);
  for (int k = 0; k < 2; ++k)
    if ((rc = LatticeOps::alloc(h, &L.d_mom[k], mom_bytes))) return rc;
  HLBM_CUDA(h, cudaMemcpyAsync(L.d_nbr, nbr.data(), nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  // rest state: delta_rho = u = S = 0 is all-zero bits in every storage
  for (int k = 0; k < 2; ++k) HLBM_CUDA(h, cudaMemsetAsync(L.d_mom[k], 0, mom_bytes, h->stream));
  if ((rc = LatticeOps::bounce(h, L))) return rc;
  if ((rc = LatticeOps::init_scales(h, L))) return rc;
  L.cur = 0;
  HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->have_blocks = true;
  ++h->hier_gen;
  return HLBM_OK;
}

int32_t hlbm_num_blocks(const hlbm_lattice* h, int32_t level, int64_t* n) {
  if (h == nullptr || n == nullptr) return HLBM_E_INVALID_ARG;
  if (level < 0 || level >= h->cfg.num_levels)
    return fail(const_cast<hlbm_lattice*>(h), HLBM_E_INVALID_ARG, "level %d out of range", level);
  *n = h->lv[level].nb;
  return HLBM_OK;
}

int32_t hlbm_get_blocks(const hlbm_lattice* h, int32_t level, int32_t* out, int64_t cap, int64_t* n,
                        uint8_t* flags_out) {
  hlbm_lattice* hm = const_cast<hlbm_lattice*>(h);
  if (h == nullptr || n == nullptr) return fail(hm, HLBM_E_INVALID_ARG, "NULL argument");
  if (level < 0 || level >= h->cfg.num_levels) return fail(hm, HLBM_E_INVALID_ARG, "level %d out of range", level);
  LevelData& L = hm->lv[level];
  *n = L.nb;
  if (cap < L.nb) return fail(hm, HLBM_E_INVALID_ARG, "capacity %lld < %lld blocks", (long long)cap, (long long)L.nb);
  if (L.nb > 0 && out == nullptr) return fail(hm, HLBM_E_INVALID_ARG, "out is NULL");
  if (!L.host_lists) {
    int rc = LatticeOps::set_device(hm);
    if (rc == HLBM_OK) rc = LatticeOps::host_lists(hm, L);
    if (rc) return rc;
  }
  if (L.nb > 0) std::memcpy(out, L.coords.data(), size_t(L.nb) * 3 * sizeof(int32_t));
  if (flags_out && L.nb > 0) std::memcpy(flags_out, L.flags.data(), size_t(L.nb));
  return HLBM_OK;
}

int32_t hlbm_set_uniform_force(hlbm_lattice* h, double fx, double fy, double fz) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (!std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(fz))
    return fail(h, HLBM_E_NONFINITE, "force is not finite");
  h->fu[0] = fx;
  h->fu[1] = fy;
  h->fu[2] = fz;
  return HLBM_OK;
}

// 1 if a device buffer (dtype 0 = f64, 1 = f32, n values) holds a non-finite
// value, 0 if not, an hlbm status (negated) on a failure.  Synchronous.
static int any_nonfinite(hlbm_lattice* h, const void* buf, int dtype, int64_t n) {
  if (h->d_count == nullptr) {
    void* p;
    if (int rc = LatticeOps::alloc(h, &p, sizeof(unsigned long long))) return -rc;
    h->d_count = static_cast<unsigned long long*>(p);
  }
  unsigned long long c = 0;
  cudaError_t e = cudaMemsetAsync(h->d_count, 0, sizeof(c), h->stream);
  if (e == cudaSuccess) e = count_nonfinite(buf, dtype, n, h->d_count, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, h->d_count, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return -fail(h, HLBM_E_CUDA, "finiteness check: %s", cudaGetErrorString(e));
  return c != 0 ? 1 : 0;
}

int32_t hlbm_set_force(hlbm_lattice* h, const float* F_dev, const float* eps_dev) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "set blocks before the force field");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  const int64_t n = h->lv[0].nb * kCells;
  int bad = F_dev ? any_nonfinite(h, F_dev, 1, n * 3) : 0;
  if (bad == 0 && eps_dev) bad = any_nonfinite(h, eps_dev, 1, n);
  if (bad < 0) return -bad;
  if (bad) return fail(h, HLBM_E_NONFINITE, "force or fluid fraction holds a non-finite value; nothing changed");
  // new fields are allocated before the old ones go: a failed call changes nothing
  void *F = nullptr, *eps = nullptr;
  if (F_dev && (rc = LatticeOps::alloc(h, &F, size_t(n) * 3 * sizeof(float)))) return rc;
  if (eps_dev && (rc = LatticeOps::alloc(h, &eps, size_t(n) * sizeof(float)))) {
    LatticeOps::release(h, F);
    return rc;
  }
  void* v = h->d_F;
  LatticeOps::release(h, v);
  v = h->d_eps;
  LatticeOps::release(h, v);
  h->d_F = static_cast<float*>(F);
  h->d_eps = static_cast<float*>(eps);
  if (F_dev)
    HLBM_CUDA(h, cudaMemcpyAsync(h->d_F, F_dev, size_t(n) * 3 * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (eps_dev)
    HLBM_CUDA(h, cudaMemcpyAsync(h->d_eps, eps_dev, size_t(n) * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return HLBM_OK;
}

int32_t hlbm_set_solid(hlbm_lattice* h, const uint8_t* mask) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (h->cfg.num_levels != 1) return fail(h, HLBM_E_UNSUPPORTED, "solid nodes need a single-level lattice");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "set blocks before the solid mask");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  LevelData& L = h->lv[0];
  void* v = L.d_solid;
  LatticeOps::release(h, v);
  L.d_solid = nullptr;
  v = L.d_bflags;
  LatticeOps::release(h, v);
  L.d_bflags = nullptr;
  if (mask == nullptr) return LatticeOps::bounce(h, L);
  if ((rc = LatticeOps::host_lists(h, L))) return rc;
  int dims[3];
  h->block_dims(0, dims);
  const int nx = h->cfg.nx, ny = h->cfg.ny;
  std::vector<uint8_t> bm(size_t(L.nb) * kCells), own(size_t(L.nb), 0), fl(size_t(L.nb), 0);
  for (int64_t b = 0; b < L.nb; ++b) {
    const int bx = L.coords[b * 3], by = L.coords[b * 3 + 1], bz = L.coords[b * 3 + 2];
    for (int c = 0; c < kCells; ++c) {
      const int x = bx * 8 + (c & 7), y = by * 8 + ((c >> 3) & 7), z = bz * 8 + (c >> 6);
      const uint8_t s = mask[(size_t(z) * ny + y) * nx + x] ? 1 : 0;
      bm[b * kCells + c] = s;
      own[b] |= s;
    }
  }
  std::vector<int32_t> nbr(size_t(L.nb) * 27);
  HLBM_CUDA(h, cudaMemcpy(nbr.data(), L.d_nbr, nbr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int64_t b = 0; b < L.nb; ++b)
    for (int d = 0; d < 27; ++d) {
      const int32_t q = nbr[b * 27 + d];
      if (q >= 0 && own[q]) fl[b] = kBlockSolidNear;
    }
  void* p;
  if ((rc = LatticeOps::alloc(h, &p, bm.size()))) return rc;
  L.d_solid = static_cast<uint8_t*>(p);
  if ((rc = LatticeOps::alloc(h, &p, fl.size()))) return rc;
  L.d_bflags = static_cast<uint8_t*>(p);
  HLBM_CUDA(h, cudaMemcpy(L.d_solid, bm.data(), bm.size(), cudaMemcpyHostToDevice));
  HLBM_CUDA(h, cudaMemcpy(L.d_bflags, fl.data(), fl.size(), cudaMemcpyHostToDevice));
  if ((rc = LatticeOps::bounce(h, L))) return rc;
  HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return HLBM_OK;
}

static int stage(hlbm_lattice* h, size_t bytes) {
  if (h->stage_bytes >= bytes) return HLBM_OK;
  LatticeOps::release(h, h->d_stage);
  h->stage_bytes = 0;
  int rc = LatticeOps::alloc(h, &h->d_stage, bytes);
  if (rc) return rc;
  h->stage_bytes = bytes;
  return HLBM_OK;
}

int32_t hlbm_write_moments(hlbm_lattice* h, int32_t level, const void* buf, int32_t dtype, int32_t on_device) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (level < 0 || level >= h->cfg.num_levels) return fail(h, HLBM_E_INVALID_ARG, "level %d out of range", level);
  if (dtype != 0 && dtype != 1) return fail(h, HLBM_E_INVALID_ARG, "dtype must be 0 (f64) or 1 (f32)");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "no blocks are stored");
  LevelData& L = h->lv[level];
  const int64_t n = L.nb * kCells;
  if (n == 0) return HLBM_OK;
  if (buf == nullptr) return fail(h, HLBM_E_INVALID_ARG, "buffer is NULL");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  const size_t bytes = size_t(n) * kRows * (dtype == 0 ? 8 : 4);
  const void* src = buf;
  if (!on_device) {
    if ((rc = stage(h, bytes))) return rc;
    HLBM_CUDA(h, cudaMemcpyAsync(h->d_stage, buf, bytes, cudaMemcpyHostToDevice, h->stream));
    src = h->d_stage;
  }
  const int bad = any_nonfinite(h, src, dtype, n * kRows);
  if (bad < 0) return -bad;
  if (bad) return fail(h, HLBM_E_NONFINITE, "moment buffer holds a non-finite value; nothing written");
  if (L.d_scales) {
    HLBM_CUDA(h, scales_from_public(src, dtype, L.nb, L.d_scales, L.d_amax, h->stream));
    L.steps_since_rescale = 0;
  }
  HLBM_CUDA(h, import_moments(h->cfg.storage, src, dtype, L.d_mom[L.cur], n, L.d_scales, h->stream));
  if (!on_device) HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return HLBM_OK;
}

int32_t hlbm_read_moments(hlbm_lattice* h, int32_t level, void* buf, int32_t dtype, int32_t on_device,
                          int32_t physical_u) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (level < 0 || level >= h->cfg.num_levels) return fail(h, HLBM_E_INVALID_ARG, "level %d out of range", level);
  if (dtype != 0 && dtype != 1) return fail(h, HLBM_E_INVALID_ARG, "dtype must be 0 (f64) or 1 (f32)");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "no blocks are stored");
  LevelData& L = h->lv[level];
  const int64_t n = L.nb * kCells;
  if (n == 0) return HLBM_OK;
  if (buf == nullptr) return fail(h, HLBM_E_INVALID_ARG, "buffer is NULL");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  const size_t bytes = size_t(n) * kRows * (dtype == 0 ? 8 : 4);
  void* dst = buf;
  if (!on_device) {
    if ((rc = stage(h, bytes))) return rc;
    dst = h->d_stage;
  }
  const bool phys = physical_u && level == 0;
  HLBM_CUDA(h, export_moments(h->cfg.storage, L.d_mom[L.cur], dst, dtype, n, L.d_scales, phys ? h->d_F : nullptr,
                              h->fu, phys ? 1 : 0, h->stream));
  if (!on_device) {
    HLBM_CUDA(h, cudaMemcpyAsync(buf, h->d_stage, bytes, cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return HLBM_OK;
}

int32_t hlbm_step(hlbm_lattice* h, int32_t n_fine_steps) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "no blocks are stored");
  const int32_t per = 1 << (h->cfg.num_levels - 1);
  if (n_fine_steps < 0 || n_fine_steps % per != 0)
    return fail(h, HLBM_E_INVALID_ARG, "n_fine_steps must be a non-negative multiple of %d", per);
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  if ((rc = LatticeOps::open_lists(h))) return rc;  // before anything is written
  if (h->device_hierarchy) return ml_advance_coarse(h, n_fine_steps / per);
  LevelData& L = h->lv[0];
  StepArgs a{};
  a.nbr = L.d_nbr;
  a.F = h->d_F;
  a.eps = h->d_eps;
  a.solid = L.d_solid;
  a.bflags = L.d_bflags;
  a.bmask = L.d_bmask;
  a.fu[0] = h->fu[0];
  a.fu[1] = h->fu[1];
  a.fu[2] = h->fu[2];
  a.tau = L.tau;
  a.om = 1.0 / L.tau;
  a.kxyz = h->cfg.xyz_literal ? 13.5 : 27.0;
  a.nb = L.nb;
  a.scales_in = a.scales_out = L.d_scales;
  for (int32_t s = 0; s < n_fine_steps; ++s) {
    a.in = L.d_mom[L.cur];
    a.out = L.d_mom[1 - L.cur];
    {
      ProfScope ps(h, kProfStreamCollide);
      if (exchange_due(h)) {  // coupled step: S, drag exchange, C (Fig. 4)
        if ((rc = coupled_step(h, a))) return rc;
        a.F = h->d_F;
      } else {
        HLBM_CUDA(h, launch_stream_collide(h->cfg.storage, a, h->stream));
      }
    }
    if (h->open_mask() != 0u) {
      ProfScope ps(h, kProfOpenFaces);
      if ((rc = open_faces_step(h, 0, a.in, a.out))) return rc;
    }
    ++h->l0_steps;
    L.cur = 1 - L.cur;
    if ((rc = LatticeOps::maybe_rescale(h, L, false))) return rc;
  }
  return HLBM_OK;
}

int32_t hlbm_synchronize(hlbm_lattice* h) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return ml_check_status(h);
}

int32_t hlbm_reduce(hlbm_lattice* h, double out[7]) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (out == nullptr) return fail(h, HLBM_E_INVALID_ARG, "out is NULL");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "no blocks are stored");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  ProfScope prof_scope(h, kProfReduce);
  size_t scratch = 0;
  for (auto& L : h->lv) scratch = std::max(scratch, reduce_scratch_doubles(L.nb));
  const size_t need = scratch + 2 * 8;
  if (h->red_n < need) {
    void* v = h->d_red;
    LatticeOps::release(h, v);
    h->d_red = nullptr;
    h->red_n = 0;
    void* p;
    if ((rc = LatticeOps::alloc(h, &p, need * sizeof(double)))) return rc;
    h->d_red = static_cast<double*>(p);
    h->red_n = need;
  }
  double* d_out = h->d_red + scratch;  // [0..4] this level, [8..15] unused
  double total[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int l = 0; l < h->cfg.num_levels; ++l) {
    LevelData& L = h->lv[l];
    if (L.nb == 0) continue;
    HLBM_CUDA(h, cudaMemsetAsync(d_out, 0, 8 * sizeof(double), h->stream));
    const double vol = std::ldexp(1.0, 3 * l);
    // the force (field or uniform) acts on level 0 only, so only level 0's
    // stored velocity carries the F / (2 rho) shift
    const double no_force[3] = {0.0, 0.0, 0.0};
    HLBM_CUDA(h, reduce_level(h->cfg.storage, L.d_mom[L.cur], L.nb, L.d_scales, L.d_skip, l == 0 ? h->d_F : nullptr,
                              l == 0 ? h->fu : no_force, vol, h->d_red, d_out, h->stream));
    double r[8];
    HLBM_CUDA(h, cudaMemcpyAsync(r, d_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 5; ++k) total[k] += r[k];
    if (l == 0)
      total[5] += r[0];
    else
      total[6] += r[0];
  }
  std::memcpy(out, total, sizeof(total));
  rc = ml_check_status(h);
  if (rc) return rc;
  if (!std::isfinite(total[0])) return fail(h, HLBM_E_NONFINITE, "mass is not finite");
  return HLBM_OK;
}

static StepArgs level0_args(hlbm_lattice* h) {
  LevelData& L = h->lv[0];
  StepArgs a{};
  a.nbr = L.d_nbr;
  a.F = h->d_F;
  a.eps = h->d_eps;
  a.solid = L.d_solid;
  a.bflags = L.d_bflags;
  a.bmask = L.d_bmask;
  for (int k = 0; k < 3; ++k) a.fu[k] = h->fu[k];
  a.tau = L.tau;
  a.om = 1.0 / L.tau;
  a.kxyz = h->cfg.xyz_literal ? 13.5 : 27.0;
  a.nb = L.nb;
  a.scales_in = a.scales_out = L.d_scales;
  return a;
}

int32_t hlbm_forward_record(hlbm_lattice* h, int32_t n_steps, int32_t ckpt_every) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (h->cfg.storage != HLBM_STORE_F32 && h->cfg.storage != HLBM_STORE_F64)
    return fail(h, HLBM_E_UNSUPPORTED, "the adjoint needs FP32 or FP64 storage");
  if (!h->have_blocks) return fail(h, HLBM_E_BAD_STATE, "no blocks are stored");
  if (n_steps <= 0 || ckpt_every <= 0) return fail(h, HLBM_E_INVALID_ARG, "n_steps and ckpt_every must be positive");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  ProfScope prof_scope(h, kProfAdjoint);
  for (void*& c : h->ckpt) LatticeOps::release(h, c);
  h->ckpt.clear();
  LatticeOps::release_tape(h);
  h->rec_steps = h->rec_every = 0;
  h->rec_gen = -1;
  if (h->drag_every > 0)
    return fail(h, HLBM_E_UNSUPPORTED, "the adjoint takes the force field as fixed: disable the live drag first");
  if (h->open_mask() != 0u) return fail(h, HLBM_E_UNSUPPORTED, "the adjoint does not cover open faces");
  auto drop = [h](int r) {  // a failed recording keeps no checkpoints and no tape
    for (void*& c : h->ckpt) LatticeOps::release(h, c);
    h->ckpt.clear();
    LatticeOps::release_tape(h);
    h->rec_steps = h->rec_every = 0;
    return r;
  };
  if (h->device_hierarchy) {  // block layout from the rebuild pipeline: the multi-level engine
    if ((rc = ml_forward_record(h, n_steps, ckpt_every))) return drop(rc);
    h->rec_gen = h->hier_gen;
    return HLBM_OK;
  }
  LevelData& L = h->lv[0];
  const size_t bytes = size_t(L.nb) * kRows * kCells * (h->cfg.storage == HLBM_STORE_F64 ? 8 : 4);
  const int n_ck = (n_steps + ckpt_every - 1) / ckpt_every;
  for (int c = 0; c < n_ck; ++c) {
    void* p;
    if ((rc = LatticeOps::alloc(h, &p, bytes))) return drop(rc);
    h->ckpt.push_back(p);
  }
  // FP32 storage: the last segment runs as the adjoint would recompute it
  // (states and pre-collision moments of every step kept as the tape; the
  // buffers are sized for a whole segment, so that the adjoint uses them for
  // every segment)
  const bool taped = h->cfg.storage == HLBM_STORE_F32;
  const int32_t t_last = (n_ck - 1) * ckpt_every;
  if (taped) {
    AdjTape* tape = new AdjTape();
    h->tape = tape;
    tape->n = n_steps - t_last;
    tape->seg.assign(size_t(ckpt_every) + 1, nullptr);
    tape->pre.assign(size_t(ckpt_every), nullptr);
    for (int i = 0; i < ckpt_every; ++i) {
      void* p = nullptr;
      if ((rc = LatticeOps::alloc(h, &p, bytes))) return drop(rc);
      tape->bufs.push_back(p);
      tape->seg[size_t(i) + 1] = p;
      if ((rc = LatticeOps::alloc(h, &p, bytes))) return drop(rc);
      tape->bufs.push_back(p);
      tape->pre[size_t(i)] = p;
    }
  }
  for (int32_t t = 0; t < n_steps; ++t) {
    if (t % ckpt_every == 0) {
      const cudaError_t e = cudaMemcpyAsync(h->ckpt[t / ckpt_every], L.d_mom[L.cur], bytes,
                                            cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) return drop(fail(h, HLBM_E_CUDA, "checkpoint copy: %s", cudaGetErrorString(e)));
    }
    if (taped && t >= t_last) break;
    if ((rc = hlbm_step(h, 1))) return drop(rc);
  }
  if (taped) {
    AdjTape* tape = h->tape;
    StepArgs a = level0_args(h);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < tape->n && e == cudaSuccess; ++i) {
      a.in = i == 0 ? h->ckpt[size_t(n_ck) - 1] : tape->seg[size_t(i)];
      a.out = tape->seg[size_t(i) + 1];
      a.pre_out = static_cast<float*>(tape->pre[size_t(i)]);
      e = launch_stream_collide_record(a, h->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(L.d_mom[L.cur], tape->seg[size_t(tape->n)], bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return drop(fail(h, HLBM_E_CUDA, "recording the last segment: %s", cudaGetErrorString(e)));
    h->l0_steps += tape->n;
  }
  h->rec_steps = n_steps;
  h->rec_every = ckpt_every;
  h->rec_gen = h->hier_gen;
  return HLBM_OK;
}

int32_t hlbm_adjoint(hlbm_lattice* h, const float* dL_dM_dev, float* dL_dF_dev) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (h->rec_steps <= 0) return fail(h, HLBM_E_BAD_STATE, "call hlbm_forward_record first");
  if (dL_dM_dev == nullptr || dL_dF_dev == nullptr) return fail(h, HLBM_E_INVALID_ARG, "NULL buffer");
  if (h->rec_gen != h->hier_gen) return fail(h, HLBM_E_BAD_STATE, "the block layout changed after hlbm_forward_record");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  ProfScope prof_scope(h, kProfAdjoint);
  if (h->device_hierarchy) return ml_adjoint(h, dL_dM_dev, dL_dF_dev);
  LevelData& L = h->lv[0];
  const int64_t nb = L.nb;
  const size_t bytes = size_t(nb) * kRows * kCells * (h->cfg.storage == HLBM_STORE_F64 ? 8 : 4);
  const size_t lam_elems = size_t(nb) * kRows * kCells;
  const int K = h->rec_every, n = h->rec_steps;
  std::vector<void*> tmp;
  auto release_all = [&]() {
    for (void*& p : tmp) LatticeOps::release(h, p);
  };
  auto get = [&](size_t b, void** out) -> int {
    int r = LatticeOps::alloc(h, out, b);
    if (r == HLBM_OK) tmp.push_back(*out);
    return r;
  };
  // FP32 storage records the pre-collision moments of every recomputed step
  // (one float32 buffer per step of a segment), so the reverse step needs no
  // second streaming pass; FP64 storage recomputes the pull in its reverse step.
  const bool record = h->cfg.storage == HLBM_STORE_F32;
  // dL/dF: an FP32 sum per checkpoint segment (dFs, FP32 storage), added to
  // the FP64 sum over segments (dF) when the segment is done
  void *lam0, *lam1, *lamp, *lamp2, *dF, *dFs = nullptr;
  std::vector<void*> seg(size_t(K) + 1, nullptr), pre(record ? size_t(K) : 0, nullptr);
  if ((rc = get(lam_elems * 4, &lam0)) || (rc = get(lam_elems * 4, &lam1)) || (rc = get(lam_elems * 4, &lamp)) ||
      (rc = get(lam_elems * 4, &lamp2)) || (rc = get(size_t(nb) * 3 * kCells * sizeof(double), &dF)) ||
      (record && (rc = get(size_t(nb) * 3 * kCells * sizeof(float), &dFs)))) {
    release_all();
    return rc;
  }
  // segment buffers: the recording's tape when there is one (it holds the
  // last segment already), else allocated here
  AdjTape* tape = record ? h->tape : nullptr;
  if (tape != nullptr) {
    for (int i = 1; i <= K; ++i) seg[size_t(i)] = tape->seg[size_t(i)];
    for (int i = 0; i < K; ++i) pre[size_t(i)] = tape->pre[size_t(i)];
  } else {
    for (int i = 1; i <= (record ? K : K - 1); ++i)
      if ((rc = get(bytes, &seg[i]))) {
        release_all();
        return rc;
      }
    for (int i = 0; i < int(pre.size()); ++i)
      if ((rc = get(lam_elems * 4, &pre[i]))) {
        release_all();
        return rc;
      }
  }
  // every allocation went through: the adjoint takes the tape over
  const bool taped = tape != nullptr;
  if (taped) {
    tmp.insert(tmp.end(), tape->bufs.begin(), tape->bufs.end());
    delete tape;
    h->tape = nullptr;
  }
  float* lam[2] = {static_cast<float*>(lam0), static_cast<float*>(lam1)};
  int c = 0;
  cudaError_t e = cudaMemcpyAsync(lam[0], dL_dM_dev, lam_elems * 4, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dF, 0, size_t(nb) * 3 * kCells * sizeof(double), h->stream);
  if (e == cudaSuccess && dFs != nullptr) e = cudaMemsetAsync(dFs, 0, size_t(nb) * 3 * kCells * sizeof(float), h->stream);
  StepArgs a = level0_args(h);
  const int n_seg = (n + K - 1) / K;
  for (int s = n_seg - 1; s >= 0 && e == cudaSuccess; --s) {
    const int t0 = s * K, ns = (n - t0) < K ? (n - t0) : K;
    seg[0] = h->ckpt[s];
    if (record) {
      // lam[0]: dL/dM of the final state (kept: solid nodes keep it for all
      // steps); lam[1]: dL/dM at the segment boundary.  Per segment: the
      // transposed collision of its last step, then for every step i > 0 its
      // reverse stream fused with the transposed collision of step i - 1, then
      // the reverse stream of the first step (not needed for the first segment:
      // only dL/dF is returned).
      float* lp[2] = {static_cast<float*>(lamp), static_cast<float*>(lamp2)};
      int q = 0;
      for (int i = 0; i < ns && e == cudaSuccess && !(taped && s == n_seg - 1); ++i) {
        // recompute the segment, keeping states and p (the last one: taped)
        a.in = seg[i];
        a.out = seg[i + 1];
        a.pre_out = static_cast<float*>(pre[i]);
        e = launch_stream_collide_record(a, h->stream);
      }
      a.pre_out = nullptr;
      a.in = seg[ns - 1];
      float* dfs = static_cast<float*>(dFs);
      if (e == cudaSuccess)
        e = adjoint_collide(a, static_cast<const float*>(pre[ns - 1]), s == n_seg - 1 ? lam[0] : lam[1], lp[q],
                            static_cast<double*>(dF), h->stream, dfs);
      for (int i = ns - 1; i >= 1 && e == cudaSuccess; --i) {
        a.in = seg[i];
        e = adjoint_push_collide(a, lp[q], static_cast<const float*>(pre[i - 1]), lp[1 - q], static_cast<double*>(dF),
                                 h->stream, nullptr, nullptr, nullptr, false, dfs);
        q = 1 - q;
      }
      if (e == cudaSuccess) e = adjoint_dF_flush(static_cast<double*>(dF), dfs, nb * 3 * kCells, h->stream);
      if (s > 0 && e == cudaSuccess) {
        a.in = seg[0];
        e = adjoint_push(a, lam[0], lp[q], lam[1], h->stream);
      }
      continue;
    }
    for (int i = 1; i < ns && e == cudaSuccess; ++i) {  // recompute the segment's states
      a.in = seg[i - 1];
      a.out = seg[i];
      e = launch_stream_collide(h->cfg.storage, a, h->stream);
    }
    for (int i = ns - 1; i >= 0 && e == cudaSuccess; --i) {
      a.in = seg[i];
      e = adjoint_step(h->cfg.storage, a, lam[c], static_cast<float*>(lamp), static_cast<double*>(dF), lam[1 - c],
                       h->stream);
      c = 1 - c;
    }
  }
  if (e == cudaSuccess) e = adjoint_dF_to_float(static_cast<double*>(dF), dL_dF_dev, nb * 3 * kCells, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  seg[0] = nullptr;
  release_all();
  if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "adjoint: %s", cudaGetErrorString(e));
  return HLBM_OK;
}

int32_t hlbm_set_profiling(hlbm_lattice* h, int32_t on) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  h->prof.on = on != 0;
  return HLBM_OK;
}

int32_t hlbm_get_profile(hlbm_lattice* h, double ms_out[8], int64_t count_out[8], int32_t reset) {
  if (h == nullptr || ms_out == nullptr || count_out == nullptr)
    return fail(h, HLBM_E_INVALID_ARG, "NULL argument");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  if ((rc = profile_collect(h))) return rc;
  for (int c = 0; c < kProfClasses; ++c) {
    ms_out[c] = h->prof.ms[c];
    count_out[c] = h->prof.count[c];
    if (reset) {
      h->prof.ms[c] = 0.0;
      h->prof.count[c] = 0;
    }
  }
  return HLBM_OK;
}

int32_t hlbm_set_block_lookup(hlbm_lattice* h, int32_t mode) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (mode != 0 && mode != 1) return fail(h, HLBM_E_INVALID_ARG, "block lookup mode must be 0 (slot table) or 1 (hash)");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  if (h->device_hierarchy && h->have_blocks) {
    // convert the stored levels now; every allocation comes first, so a failed
    // call leaves the levels as they were
    const int L = h->cfg.num_levels;
    std::vector<void*> a(size_t(2 * L), nullptr);
    std::vector<uint32_t> cap(size_t(L), 0);
    auto undo = [&](int r) {
      for (void*& p : a) LatticeOps::release(h, p);
      return r;
    };
    for (int l = 0; l < L; ++l) {
      LevelData& X = h->lv[l];
      int dims[3];
      h->block_dims(l, dims);
      const GridDims d{dims[0], dims[1], dims[2]};
      if (mode == 1 && X.d_hkeys == nullptr && X.nb > 0) {
        cap[size_t(l)] = hash_capacity(X.nb);
        if ((rc = LatticeOps::alloc(h, &a[size_t(2 * l)], cap[size_t(l)] * sizeof(unsigned long long))) ||
            (rc = LatticeOps::alloc(h, &a[size_t(2 * l + 1)], cap[size_t(l)] * sizeof(int32_t))))
          return undo(rc);
      } else if (mode == 0 && X.d_slot == nullptr) {
        if ((rc = LatticeOps::alloc(h, &a[size_t(2 * l)], size_t(d.slots()) * sizeof(int32_t)))) return undo(rc);
      }
    }
    for (int l = 0; l < L; ++l) {
      LevelData& X = h->lv[l];
      int dims[3];
      h->block_dims(l, dims);
      const GridDims d{dims[0], dims[1], dims[2]};
      cudaError_t e = cudaSuccess;
      if (mode == 1 && a[size_t(2 * l)] != nullptr) {
        X.d_hkeys = static_cast<unsigned long long*>(a[size_t(2 * l)]);
        X.d_hvals = static_cast<int32_t*>(a[size_t(2 * l + 1)]);
        X.hcap = cap[size_t(l)];
        a[size_t(2 * l)] = a[size_t(2 * l + 1)] = nullptr;
        e = build_block_hash(X.d_coords, X.nb, X.d_hkeys, X.d_hvals, X.hcap, h->stream);
        void* v = X.d_slot;
        LatticeOps::release(h, v);
        X.d_slot = nullptr;
      } else if (mode == 0 && a[size_t(2 * l)] != nullptr) {
        X.d_slot = static_cast<int32_t*>(a[size_t(2 * l)]);
        a[size_t(2 * l)] = nullptr;
        e = slot_table(X.d_coords, X.nb, d, X.d_slot, h->stream);
        void* v = X.d_hkeys;
        LatticeOps::release(h, v);
        X.d_hkeys = nullptr;
        v = X.d_hvals;
        LatticeOps::release(h, v);
        X.d_hvals = nullptr;
        X.hcap = 0;
      }
      if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "block lookup: %s", cudaGetErrorString(e));
    }
    HLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  h->block_lookup = mode;
  return HLBM_OK;
}

int32_t hlbm_get_block_lookup(const hlbm_lattice* h, int32_t* mode, int64_t* table_bytes) {
  hlbm_lattice* hm = const_cast<hlbm_lattice*>(h);
  if (h == nullptr || mode == nullptr || table_bytes == nullptr) return fail(hm, HLBM_E_INVALID_ARG, "NULL argument");
  *mode = h->block_lookup;
  int64_t bytes = 0;
  for (int l = 0; l < h->cfg.num_levels; ++l) {
    const LevelData& X = h->lv[l];
    int dims[3];
    h->block_dims(l, dims);
    if (X.d_slot != nullptr) bytes += int64_t(dims[0]) * dims[1] * dims[2] * int64_t(sizeof(int32_t));
    if (X.d_hkeys != nullptr) bytes += int64_t(X.hcap) * int64_t(sizeof(unsigned long long) + sizeof(int32_t));
  }
  *table_bytes = bytes;
  return HLBM_OK;
}

int32_t hlbm_test_narrow(const double* in_dev, float* out_dev, float* hw_dev, int64_t n) {
  if (n < 0 || (n > 0 && (in_dev == nullptr || out_dev == nullptr || hw_dev == nullptr)))
    return fail(nullptr, HLBM_E_INVALID_ARG, "bad buffers");
  cudaError_t e = test_narrow(in_dev, out_dev, hw_dev, n, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(nullptr, HLBM_E_CUDA, "narrowing test: %s", cudaGetErrorString(e));
  return HLBM_OK;
}

int32_t hlbm_inject_alloc_failure(int64_t after) {
  g_alloc_fail_after.store(after < 0 ? -1 : after);
  return HLBM_OK;
}

int32_t hlbm_set_fine_blocks(hlbm_lattice* h, const int32_t* coords_xyz, int64_t n) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (n < 0 || (n > 0 && coords_xyz == nullptr)) return fail(h, HLBM_E_INVALID_ARG, "bad block list");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  int dims[3];
  h->block_dims(0, dims);
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a)
      if (coords_xyz[3 * i + a] < 0 || coords_xyz[3 * i + a] >= dims[a])
        return fail(h, HLBM_E_INVALID_ARG, "block %lld coordinate %d = %d outside [0, %d)", (long long)i, a,
                    coords_xyz[3 * i + a], dims[a]);
  return ml_rebuild(h, nullptr, 0, 0, coords_xyz, n, nullptr);
}

int32_t hlbm_set_blocks(hlbm_lattice* h, int32_t level, const int32_t* coords_xyz, int64_t n) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (level < 0 || level >= h->cfg.num_levels) return fail(h, HLBM_E_INVALID_ARG, "level %d out of range", level);
  if (n < 0 || (n > 0 && coords_xyz == nullptr)) return fail(h, HLBM_E_INVALID_ARG, "bad block list");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  return ml_set_blocks(h, level, coords_xyz, n);
}

int32_t hlbm_rebuild_from_particles(hlbm_lattice* h, const float* pos_xyz, int64_t n, int32_t on_device,
                                    int64_t counts_out[3]) {
  if (h == nullptr) return fail(nullptr, HLBM_E_INVALID_ARG, "handle is NULL");
  if (n < 0 || (n > 0 && pos_xyz == nullptr)) return fail(h, HLBM_E_INVALID_ARG, "bad particle buffer");
  int rc = LatticeOps::set_device(h);
  if (rc) return rc;
  return ml_rebuild(h, pos_xyz, n, on_device, nullptr, 0, counts_out);
}

int32_t hlbm_get_interface_nodes(const hlbm_lattice* h, int32_t level, int32_t which, int32_t* out, int64_t cap,
                                 int64_t* n) {
  hlbm_lattice* hm = const_cast<hlbm_lattice*>(h);
  if (h == nullptr || n == nullptr) return fail(hm, HLBM_E_INVALID_ARG, "NULL argument");
  if (level < 0 || level >= h->cfg.num_levels) return fail(hm, HLBM_E_INVALID_ARG, "level %d out of range", level);
  if (which != 0 && which != 1) return fail(hm, HLBM_E_INVALID_ARG, "which must be 0 (down) or 1 (up)");
  const LevelData& L = h->lv[level];
  const int64_t cnt = which == 0 ? L.n_down : L.n_up;
  *n = cnt;
  if (cap < cnt) return fail(hm, HLBM_E_INVALID_ARG, "capacity %lld < %lld nodes", (long long)cap, (long long)cnt);
  if (cnt == 0) return HLBM_OK;
  if (out == nullptr) return fail(hm, HLBM_E_INVALID_ARG, "out is NULL");
  int rc = LatticeOps::set_device(hm);
  if (rc) return rc;
  HLBM_CUDA(hm, cudaMemcpy(out, which == 0 ? L.d_down : L.d_up, size_t(cnt) * sizeof(int32_t),
                           cudaMemcpyDeviceToHost));
  return HLBM_OK;
}

}  // extern "C"

// Records the message returned by hlbm_last_error(NULL) for entry points that
// take no handle.
void hlbm_internal_set_error(const char* msg) { g_create_error = msg ? msg : ""; }
