// batch.cu -- many independent single-level periodic domains advanced together.
//
// The stored blocks of every domain are concatenated into one flattened list
// (domain-major, slot order inside a domain); each block's neighbour table
// wraps inside its own domain, each block carries its domain's 1/tau and the
// index of its domain's row scales.  The stream-collide kernel is the
// single-lattice one: one launch advances every domain.  The
// launch strategies:
//   HLBM_BATCH_ONE_LAUNCH        one launch per step, one CTA per block
//   HLBM_BATCH_GRAPH             the same, kBatchGraphSteps steps captured in a CUDA graph
//   HLBM_BATCH_PER_DOMAIN        one launch per domain per step (block sub-ranges)
//   HLBM_BATCH_PERSISTENT        one launch per step of resident CTAs that take
//                                blocks from an atomic ticket counter
//   HLBM_BATCH_PERSISTENT_GRAPH  the same, captured in a CUDA graph
// hlbm_batch_autotune times the strategies and keeps the fastest.
#include <cuda_runtime.h>

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

namespace {
constexpr int kBatchGraphSteps = 32;  // = the rescale period, so a graph ends on a refit
}

struct hlbm_batch {
  int n_dom = 0;
  int storage = HLBM_STORE_F32;
  int xyz_literal = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  std::vector<int32_t> ext;        // [n_dom][3]
  std::vector<double> tau;         // [n_dom]
  std::vector<int64_t> begin;      // [n_dom + 1] block ranges
  int64_t nb = 0;
  int32_t* d_nbr = nullptr;
  void* d_mom[2] = {nullptr, nullptr};
  int cur = 0;
  float* d_om = nullptr;
  int32_t* d_dom = nullptr;
  uint8_t* d_bflags = nullptr;
  uint32_t* d_bmask = nullptr;
  hlbm::Scales* d_scales = nullptr;  // [n_dom]
  hlbm::Scales* d_tmp = nullptr;     // [n_dom]
  unsigned* d_amax = nullptr;        // [n_dom][10]
  int steps_since_rescale = 0;
  int mode = HLBM_BATCH_GRAPH;
  cudaGraphExec_t graph = nullptr;
  int graph_cur = -1;   // buffer parity the graph was captured at
  int graph_mode = -1;  // strategy the graph was captured with
  unsigned* d_work = nullptr;  // ticket counter of the persistent kernel
  int persistent_grid = 0;
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(hlbm_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b)
    b->err = buf;
  else
    g_batch_error = buf;
  return code;
}

#define B_CUDA(b, call)                                                                          \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return bfail((b), HLBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
int balloc(hlbm_batch* b, P** p, size_t count) {
  *p = nullptr;
  if (count == 0) return HLBM_OK;
  if (hlbm::alloc_failure_injected())
    return bfail(b, HLBM_E_OOM, "allocation of %zu bytes failed (injected)", count * sizeof(P));
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(P));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, HLBM_E_OOM, "cudaMalloc(%zu): %s", count * sizeof(P), cudaGetErrorString(e));
  }
  *p = static_cast<P*>(v);
  return HLBM_OK;
}

size_t elem_bytes(int storage) { return storage == HLBM_STORE_F64 ? 8 : (storage == HLBM_STORE_F32 ? 4 : 2); }
bool reduced(int storage) { return storage == HLBM_STORE_F16S || storage == HLBM_STORE_BF16S; }

hlbm::StepArgs batch_args(hlbm_batch* b) {
  hlbm::StepArgs a{};
  a.nbr = b->d_nbr;
  a.bflags = b->d_bflags;
  a.bmask = b->d_bmask;
  a.kxyz = b->xyz_literal ? 13.5 : 27.0;
  a.nb = b->nb;
  a.blk0 = 0;
  a.blk_om = b->d_om;
  a.blk_dom = b->d_dom;
  a.scales_in = a.scales_out = b->d_scales;
  a.tau = 1.0;
  a.om = 1.0;
  return a;
}

bool is_graph(int mode) { return mode == HLBM_BATCH_GRAPH || mode == HLBM_BATCH_PERSISTENT_GRAPH; }
bool is_persistent(int mode) { return mode == HLBM_BATCH_PERSISTENT || mode == HLBM_BATCH_PERSISTENT_GRAPH; }

// One step with the given strategy (no graph), then the periodic refit.
int step_direct(hlbm_batch* b, int mode) {
  hlbm::StepArgs a = batch_args(b);
  a.in = b->d_mom[b->cur];
  a.out = b->d_mom[1 - b->cur];
  if (is_persistent(mode)) {
    a.work = b->d_work;
    a.grid = int(std::min<int64_t>(b->persistent_grid, b->nb));
  }
  if (mode == HLBM_BATCH_PER_DOMAIN) {
    for (int d = 0; d < b->n_dom; ++d) {
      a.blk0 = b->begin[d];
      a.nb = b->begin[d + 1] - b->begin[d];
      B_CUDA(b, hlbm::launch_stream_collide(b->storage, a, b->stream));
    }
  } else {
    B_CUDA(b, hlbm::launch_stream_collide(b->storage, a, b->stream));
  }
  b->cur = 1 - b->cur;
  if (reduced(b->storage) && ++b->steps_since_rescale >= hlbm::kRescaleEvery) {
    b->steps_since_rescale = 0;
    if (mode == HLBM_BATCH_PER_DOMAIN) {  // as separate lattices would
      const size_t eb = elem_bytes(b->storage);
      for (int d = 0; d < b->n_dom; ++d) {
        char* base = static_cast<char*>(b->d_mom[b->cur]) + size_t(b->begin[d]) * hlbm::kRows * hlbm::kCells * eb;
        B_CUDA(b, hlbm::rescale_storage(b->storage, base, b->begin[d + 1] - b->begin[d], b->d_scales + d,
                                        b->d_tmp + d, b->d_amax + d * hlbm::kRows, b->stream));
      }
    } else {  // every domain's refit in three launches
      B_CUDA(b, hlbm::rescale_storage_domains(b->storage, b->d_mom[b->cur], b->nb, b->d_dom, b->n_dom, b->d_scales,
                                              b->d_tmp, b->d_amax, b->stream));
    }
  }
  return HLBM_OK;
}

void drop_graph(hlbm_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_cur = -1;
  b->graph_mode = -1;
}

int build_graph(hlbm_batch* b) {
  drop_graph(b);
  const int cur0 = b->cur, since0 = b->steps_since_rescale;
  b->steps_since_rescale = 0;  // the graph's refit lands on its last step
  B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = HLBM_OK;
  for (int s = 0; s < kBatchGraphSteps && rc == HLBM_OK; ++s) rc = step_direct(b, b->mode);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  b->cur = cur0;
  b->steps_since_rescale = since0;
  if (rc != HLBM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, HLBM_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, HLBM_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  b->graph_cur = cur0;
  b->graph_mode = b->mode;
  return HLBM_OK;
}

int stage(hlbm_batch* b, size_t bytes) {
  if (b->stage_bytes >= bytes) return HLBM_OK;
  if (b->d_stage) cudaFree(b->d_stage);
  b->d_stage = nullptr;
  b->stage_bytes = 0;
  char* p = nullptr;
  int rc = balloc(b, &p, bytes);
  if (rc) return rc;
  b->d_stage = p;
  b->stage_bytes = bytes;
  return HLBM_OK;
}

}  // namespace

extern "C" {

const char* hlbm_batch_last_error(const hlbm_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

int32_t hlbm_batch_destroy(hlbm_batch* b) {
  if (b == nullptr) return HLBM_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (void* p : {(void*)b->d_nbr, b->d_mom[0], b->d_mom[1], (void*)b->d_om, (void*)b->d_dom, (void*)b->d_bflags,
                  (void*)b->d_bmask, (void*)b->d_scales, (void*)b->d_tmp, (void*)b->d_amax, b->d_stage,
                  (void*)b->d_work})
    if (p) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return HLBM_OK;
}

int32_t hlbm_batch_create(const hlbm_config* cfgs, int32_t n, hlbm_batch** out) {
  if (out == nullptr) return bfail(nullptr, HLBM_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (cfgs == nullptr || n <= 0) return bfail(nullptr, HLBM_E_INVALID_ARG, "need at least one domain");
  const hlbm_config& c0 = cfgs[0];
  if (c0.storage == HLBM_STORE_F64 || c0.storage < 0 || c0.storage > HLBM_STORE_BF16S)
    return bfail(nullptr, HLBM_E_UNSUPPORTED, "batches use FP32, FP16S or BF16S storage");
  for (int d = 0; d < n; ++d) {
    const hlbm_config& c = cfgs[d];
    if (c.num_levels != 1 || c.block_edge != 8 || !c.periodic[0] || !c.periodic[1] || !c.periodic[2])
      return bfail(nullptr, HLBM_E_INVALID_ARG, "domain %d: batches hold single-level periodic domains of 8^3 blocks", d);
    if (c.storage != c0.storage || c.device != c0.device || c.stream != c0.stream)
      return bfail(nullptr, HLBM_E_INVALID_ARG, "domain %d: storage, device and stream must match domain 0", d);
    if (c.nx <= 0 || c.ny <= 0 || c.nz <= 0 || c.nx % 8 || c.ny % 8 || c.nz % 8)
      return bfail(nullptr, HLBM_E_INVALID_ARG, "domain %d: extents must be positive multiples of 8", d);
    if (!(c.tau_finest > 0.5) || !std::isfinite(c.tau_finest))
      return bfail(nullptr, HLBM_E_INVALID_ARG, "domain %d: tau must exceed 1/2", d);
  }
  hlbm_batch* b = new (std::nothrow) hlbm_batch();
  if (b == nullptr) return bfail(nullptr, HLBM_E_OOM, "host allocation failed");
  b->n_dom = n;
  b->storage = c0.storage;
  b->xyz_literal = c0.xyz_literal;
  b->device = c0.device;
  if (cudaSetDevice(b->device) != cudaSuccess) {
    delete b;
    return bfail(nullptr, HLBM_E_CUDA, "cudaSetDevice(%d) failed", c0.device);
  }
  b->stream = static_cast<cudaStream_t>(c0.stream);
  if (b->stream == nullptr) {  // graphs need a capturable stream
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return bfail(nullptr, HLBM_E_CUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  b->begin.assign(size_t(n) + 1, 0);
  for (int d = 0; d < n; ++d) {
    b->ext.insert(b->ext.end(), {cfgs[d].nx, cfgs[d].ny, cfgs[d].nz});
    b->tau.push_back(cfgs[d].tau_finest);
    b->begin[d + 1] = b->begin[d] + int64_t(cfgs[d].nx / 8) * (cfgs[d].ny / 8) * (cfgs[d].nz / 8);
  }
  b->nb = b->begin[n];
  // host tables: neighbours (wrapping inside each domain), 1/tau, domain index
  std::vector<int32_t> nbr(size_t(b->nb) * 27);
  std::vector<float> om(size_t(b->nb));
  std::vector<int32_t> dom(size_t(b->nb));
  for (int d = 0; d < n; ++d) {
    const int bx = b->ext[3 * d] / 8, by = b->ext[3 * d + 1] / 8, bz = b->ext[3 * d + 2] / 8;
    for (int64_t s = 0; s < b->begin[d + 1] - b->begin[d]; ++s) {
      const int x = int(s % bx), y = int((s / bx) % by), z = int(s / (int64_t(bx) * by));
      const int64_t g = b->begin[d] + s;
      om[g] = float(1.0 / b->tau[d]);
      dom[g] = d;
      for (int k = 0; k < 27; ++k) {
        const int qx = (x + k % 3 - 1 + bx) % bx, qy = (y + (k / 3) % 3 - 1 + by) % by,
                  qz = (z + k / 9 - 1 + bz) % bz;
        nbr[g * 27 + k] = int32_t(b->begin[d] + (int64_t(qz) * by + qy) * bx + qx);
      }
    }
  }
  int rc = HLBM_OK;
  const size_t mom_bytes = size_t(b->nb) * hlbm::kRows * hlbm::kCells * elem_bytes(b->storage);
  char *m0 = nullptr, *m1 = nullptr;
  if ((rc = balloc(b, &b->d_nbr, nbr.size())) || (rc = balloc(b, &m0, mom_bytes)) || (rc = balloc(b, &m1, mom_bytes)) ||
      (rc = balloc(b, &b->d_om, om.size())) || (rc = balloc(b, &b->d_dom, dom.size())) ||
      (rc = balloc(b, &b->d_bflags, size_t(b->nb))) || (rc = balloc(b, &b->d_bmask, size_t(b->nb) * hlbm::kCells)) ||
      (rc = balloc(b, &b->d_work, 2))) {
    g_batch_error = b->err;
    b->d_mom[0] = m0;
    b->d_mom[1] = m1;
    hlbm_batch_destroy(b);
    return rc;
  }
  b->d_mom[0] = m0;
  b->d_mom[1] = m1;
  cudaError_t e = cudaMemcpy(b->d_nbr, nbr.data(), nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_om, om.data(), om.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_dom, dom.data(), dom.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_bflags, 0, size_t(b->nb));
  if (e == cudaSuccess) e = cudaMemset(b->d_work, 0, 2 * sizeof(unsigned));
  if (e == cudaSuccess) {
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = hlbm::persistent_ctas_per_sm(b->storage, &per_sm);
    b->persistent_grid = std::max(1, sms * per_sm);
  }
  if (e == cudaSuccess) e = cudaMemset(m0, 0, mom_bytes);
  if (e == cudaSuccess) e = cudaMemset(m1, 0, mom_bytes);
  if (e == cudaSuccess) e = hlbm::compute_bounce_masks(b->d_nbr, nullptr, b->d_bflags, b->d_bmask, b->nb, b->stream);
  if (e == cudaSuccess && reduced(b->storage)) {
    if ((rc = balloc(b, &b->d_scales, size_t(n))) || (rc = balloc(b, &b->d_tmp, size_t(n))) ||
        (rc = balloc(b, &b->d_amax, size_t(n) * hlbm::kRows))) {
      g_batch_error = b->err;
      hlbm_batch_destroy(b);
      return rc;
    }
    for (int d = 0; d < n && e == cudaSuccess; ++d)
      e = hlbm::scales_from_public(nullptr, 1, 0, b->d_scales + d, b->d_amax + d * hlbm::kRows, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    bfail(nullptr, HLBM_E_CUDA, "batch set-up: %s", cudaGetErrorString(e));
    hlbm_batch_destroy(b);
    return HLBM_E_CUDA;
  }
  *out = b;
  return HLBM_OK;
}

int32_t hlbm_batch_num_blocks(const hlbm_batch* b, int32_t domain, int64_t* n) {
  if (b == nullptr || n == nullptr || domain < -1 || domain >= b->n_dom) return HLBM_E_INVALID_ARG;
  *n = domain < 0 ? b->nb : b->begin[domain + 1] - b->begin[domain];
  return HLBM_OK;
}

int32_t hlbm_batch_write_moments(hlbm_batch* b, int32_t domain, const void* buf, int32_t dtype, int32_t on_device) {
  if (b == nullptr) return bfail(nullptr, HLBM_E_INVALID_ARG, "batch is NULL");
  if (domain < 0 || domain >= b->n_dom) return bfail(b, HLBM_E_INVALID_ARG, "domain %d out of range", domain);
  if ((dtype != 0 && dtype != 1) || buf == nullptr) return bfail(b, HLBM_E_INVALID_ARG, "bad buffer or dtype");
  B_CUDA(b, cudaSetDevice(b->device));
  const int64_t nbd = b->begin[domain + 1] - b->begin[domain];
  const size_t bytes = size_t(nbd) * hlbm::kRows * hlbm::kCells * (dtype == 0 ? 8 : 4);
  const void* src = buf;
  int rc;
  if (!on_device) {
    if ((rc = stage(b, bytes))) return rc;
    B_CUDA(b, cudaMemcpyAsync(b->d_stage, buf, bytes, cudaMemcpyHostToDevice, b->stream));
    src = b->d_stage;
  }
  hlbm::Scales* sc = b->d_scales ? b->d_scales + domain : nullptr;
  if (sc) B_CUDA(b, hlbm::scales_from_public(src, dtype, nbd, sc, b->d_amax + domain * hlbm::kRows, b->stream));
  char* dst = static_cast<char*>(b->d_mom[b->cur]) + size_t(b->begin[domain]) * hlbm::kRows * hlbm::kCells *
                                                         elem_bytes(b->storage);
  B_CUDA(b, hlbm::import_moments(b->storage, src, dtype, dst, nbd * hlbm::kCells, sc, b->stream));
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  return HLBM_OK;
}

int32_t hlbm_batch_read_moments(hlbm_batch* b, int32_t domain, void* buf, int32_t dtype, int32_t on_device) {
  if (b == nullptr) return bfail(nullptr, HLBM_E_INVALID_ARG, "batch is NULL");
  if (domain < 0 || domain >= b->n_dom) return bfail(b, HLBM_E_INVALID_ARG, "domain %d out of range", domain);
  if ((dtype != 0 && dtype != 1) || buf == nullptr) return bfail(b, HLBM_E_INVALID_ARG, "bad buffer or dtype");
  B_CUDA(b, cudaSetDevice(b->device));
  const int64_t nbd = b->begin[domain + 1] - b->begin[domain];
  const size_t bytes = size_t(nbd) * hlbm::kRows * hlbm::kCells * (dtype == 0 ? 8 : 4);
  void* dst = buf;
  int rc;
  if (!on_device) {
    if ((rc = stage(b, bytes))) return rc;
    dst = b->d_stage;
  }
  const char* src = static_cast<const char*>(b->d_mom[b->cur]) +
                    size_t(b->begin[domain]) * hlbm::kRows * hlbm::kCells * elem_bytes(b->storage);
  const double fu[3] = {0, 0, 0};
  B_CUDA(b, hlbm::export_moments(b->storage, src, dst, dtype, nbd * hlbm::kCells,
                                 b->d_scales ? b->d_scales + domain : nullptr, nullptr, fu, 0, b->stream));
  if (!on_device) B_CUDA(b, cudaMemcpyAsync(buf, b->d_stage, bytes, cudaMemcpyDeviceToHost, b->stream));
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  return HLBM_OK;
}

int32_t hlbm_batch_step(hlbm_batch* b, int32_t n_steps) {
  if (b == nullptr) return bfail(nullptr, HLBM_E_INVALID_ARG, "batch is NULL");
  if (n_steps < 0) return bfail(b, HLBM_E_INVALID_ARG, "n_steps must be non-negative");
  B_CUDA(b, cudaSetDevice(b->device));
  int rc;
  int32_t left = n_steps;
  if (is_graph(b->mode)) {
    // run direct steps up to the next refit boundary, then whole graphs
    while (left > 0 && b->steps_since_rescale != 0) {
      if ((rc = step_direct(b, b->mode))) return rc;
      --left;
    }
    while (left >= kBatchGraphSteps) {
      if (b->graph == nullptr || b->graph_cur != b->cur || b->graph_mode != b->mode)
        if ((rc = build_graph(b))) return rc;
      B_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
      left -= kBatchGraphSteps;  // kBatchGraphSteps is even: the parity is unchanged
    }
  }
  for (; left > 0; --left)
    if ((rc = step_direct(b, b->mode))) return rc;
  return HLBM_OK;
}

int32_t hlbm_batch_synchronize(hlbm_batch* b) {
  if (b == nullptr) return bfail(nullptr, HLBM_E_INVALID_ARG, "batch is NULL");
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  return HLBM_OK;
}

int32_t hlbm_batch_set_mode(hlbm_batch* b, int32_t mode) {
  if (b == nullptr) return bfail(nullptr, HLBM_E_INVALID_ARG, "batch is NULL");
  if (mode < HLBM_BATCH_ONE_LAUNCH || mode > HLBM_BATCH_PERSISTENT_GRAPH)
    return bfail(b, HLBM_E_INVALID_ARG, "unknown mode %d", mode);
  b->mode = mode;
  return HLBM_OK;
}

int32_t hlbm_batch_autotune(hlbm_batch* b, int32_t trial_steps, int32_t* mode_out, float* ms_out) {
  if (b == nullptr) return bfail(nullptr, HLBM_E_INVALID_ARG, "batch is NULL");
  if (trial_steps < 2 * kBatchGraphSteps) trial_steps = 2 * kBatchGraphSteps;
  B_CUDA(b, cudaSetDevice(b->device));
  // the trial steps run on a copy of the state, which is restored afterwards
  const size_t mom_bytes = size_t(b->nb) * hlbm::kRows * hlbm::kCells * elem_bytes(b->storage);
  // (moment codes and, for reduced precision, the row scales they are coded with)
  const size_t sc_bytes = b->d_scales ? size_t(b->n_dom) * sizeof(hlbm::Scales) : 0;
  char* save = nullptr;
  int rc = balloc(b, &save, mom_bytes + sc_bytes);
  if (rc) return rc;
  B_CUDA(b, cudaMemcpyAsync(save, b->d_mom[b->cur], mom_bytes, cudaMemcpyDeviceToDevice, b->stream));
  if (sc_bytes)
    B_CUDA(b, cudaMemcpyAsync(save + mom_bytes, b->d_scales, sc_bytes, cudaMemcpyDeviceToDevice, b->stream));
  const int cur0 = b->cur, since0 = b->steps_since_rescale;
  cudaEvent_t e0, e1;
  B_CUDA(b, cudaEventCreate(&e0));
  B_CUDA(b, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_mode = HLBM_BATCH_ONE_LAUNCH;
  for (int mode = HLBM_BATCH_ONE_LAUNCH; mode <= HLBM_BATCH_PERSISTENT_GRAPH && rc == HLBM_OK; ++mode) {
    b->mode = mode;
    b->steps_since_rescale = 0;
    if ((rc = hlbm_batch_step(b, kBatchGraphSteps))) break;  // warm-up (and graph build)
    cudaEventRecord(e0, b->stream);
    if ((rc = hlbm_batch_step(b, trial_steps))) break;
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= float(trial_steps);
    if (ms_out) ms_out[mode] = ms;
    if (ms < best) {
      best = ms;
      best_mode = mode;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the state the trials started from
  b->cur = cur0;
  b->steps_since_rescale = since0;
  cudaMemcpyAsync(b->d_mom[b->cur], save, mom_bytes, cudaMemcpyDeviceToDevice, b->stream);
  if (sc_bytes) cudaMemcpyAsync(b->d_scales, save + mom_bytes, sc_bytes, cudaMemcpyDeviceToDevice, b->stream);
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  if (rc) return rc;
  b->mode = best_mode;
  if (mode_out) *mode_out = best_mode;
  return HLBM_OK;
}

}  // extern "C"
