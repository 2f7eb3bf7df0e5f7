// ml_host.cu -- host orchestration of the multi-level engine: the rebuild
// pipeline of Sec. 6.3 (occupancy -> Phi -> sets -> compaction -> tables ->
// interface lists -> moments of the new blocks) and the sub-cycled advance of
// Algorithm 1 with its downward and upward transfers.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "hierarchy.cuh"
#include "hlbm_internal.h"
#include "lattice_state.h"
#include "multilevel.cuh"

namespace hlbm {
namespace {

#define ML_CUDA(h, call)                                                                       \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail((h), HLBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define ML_TRY(expr)        \
  do {                      \
    int rc_ = (expr);       \
    if (rc_ != HLBM_OK) return rc_; \
  } while (0)

size_t storage_size(int storage) { return storage == HLBM_STORE_F64 ? 8 : (storage == HLBM_STORE_F32 ? 4 : 2); }

GridDims dims_of(const hlbm_lattice* h, int l) {
  int d[3];
  h->block_dims(l, d);
  return GridDims{d[0], d[1], d[2]};
}

template <typename P>
int alloc_t(hlbm_lattice* h, P** p, size_t count) {
  void* v = nullptr;
  int rc = LatticeOps::alloc(h, &v, count * sizeof(P));
  *p = static_cast<P*>(v);
  return rc;
}

LevelView view_of(const LevelData& L, GridDims d) {
  LevelView v;
  v.d = d;
  v.slot = L.d_slot;
  v.hash = BlockHash{L.d_hkeys, L.d_hvals, L.hcap ? L.hcap - 1u : 0u};
  v.coords = L.d_coords;
  v.mom = L.d_mom[L.cur];
  v.mom_other = L.d_mom[1 - L.cur];
  v.nb = L.nb;
  v.sc = L.d_scales;
  return v;
}

// Transfers of Algorithm 1 ------------------------------------------------------

int downward(hlbm_lattice* h, int l, int s, bool refresh) {
  ProfScope prof_scope(h, kProfDown);
  LevelData& F = h->lv[l];
  LevelData& C = h->lv[l + 1];
  if (F.n_down == 0) return HLBM_OK;
  TransferArgs a{};
  a.fine = view_of(F, dims_of(h, l));
  a.coarse = view_of(C, dims_of(h, l + 1));
  a.out = F.d_mom[F.cur];
  a.out_sc = F.d_scales;
  a.nodes = F.d_down_t;
  a.stencil = F.d_down_stc;
  a.n_nodes = F.n_down;
  a.avg = (!refresh && s == 2) ? 1 : 0;
  a.use_other = (!refresh && s == 1) ? 1 : 0;
  a.acc_old = refresh ? nullptr : F.d_down_acc;
  a.k = h->kdown[l];
  for (int ax = 0; ax < 3; ++ax) a.periodic[ax] = h->cfg.periodic[ax];
  a.status = h->d_status;
  ML_CUDA(h, transfer_down(h->cfg.storage, a, h->stream));
  return HLBM_OK;
}

int upward(hlbm_lattice* h, int l) {
  ProfScope prof_scope(h, kProfUp);
  LevelData& F = h->lv[l];
  LevelData& C = h->lv[l + 1];
  if (C.n_up == 0) return HLBM_OK;
  TransferArgs a{};
  a.fine = view_of(F, dims_of(h, l));
  a.coarse = view_of(C, dims_of(h, l + 1));
  a.out = C.d_mom[C.cur];
  a.out_sc = C.d_scales;
  a.nodes = C.d_up;
  a.n_nodes = C.n_up;
  a.k = h->kup[l];
  for (int ax = 0; ax < 3; ++ax) a.periodic[ax] = h->cfg.periodic[ax];
  a.status = h->d_status;
  ML_CUDA(h, transfer_up(h->cfg.storage, a, h->stream));
  return HLBM_OK;
}

int streaming_collision(hlbm_lattice* h, int l) {
  LevelData& L = h->lv[l];
  if (L.nb == 0) {
    L.cur = 1 - L.cur;
    return HLBM_OK;
  }
  StepArgs a{};
  a.in = L.d_mom[L.cur];
  a.out = L.d_mom[1 - L.cur];
  a.nbr = L.d_nbr;
  a.F = l == 0 ? h->d_F : nullptr;
  a.eps = l == 0 ? h->d_eps : nullptr;
  a.solid = L.d_solid;
  a.bflags = L.d_bflags;
  a.bmask = L.d_bmask;
  for (int ax = 0; ax < 3; ++ax) a.fu[ax] = l == 0 ? h->fu[ax] : 0.0;
  a.tau = L.tau;
  a.om = 1.0 / L.tau;
  a.kxyz = h->cfg.xyz_literal ? 13.5 : 27.0;
  a.nb = L.nb;
  a.scales_in = a.scales_out = L.d_scales;
  {
    ProfScope prof_scope(h, kProfStreamCollide);
    if (l == 0 && exchange_due(h)) {  // coupled step: S, drag exchange, C (Fig. 4)
      ML_TRY(coupled_step(h, a));
    } else {
      ML_CUDA(h, launch_stream_collide(h->cfg.storage, a, h->stream));
    }
  }
  if (h->open_mask() != 0u) {
    ProfScope prof_scope(h, kProfOpenFaces);
    ML_TRY(open_faces_step(h, l, a.in, a.out));
  }
  if (l == 0) ++h->l0_steps;
  L.cur = 1 - L.cur;
  return LatticeOps::maybe_rescale(h, L, false);
}

// AdvanceLBM(l, s) of Algorithm 1.
int advance(hlbm_lattice* h, int l, int s) {
  const int L = h->cfg.num_levels;
  if (l < L - 1) ML_TRY(downward(h, l, s, false));
  ML_TRY(streaming_collision(h, l));
  if (l < L - 1 && s == 2) ML_TRY(upward(h, l));
  if (l > 0) {
    ML_TRY(advance(h, l - 1, 1));
    ML_TRY(advance(h, l - 1, 2));
  }
  return HLBM_OK;
}

}  // namespace

int ml_advance_coarse(hlbm_lattice* h, int64_t n_coarse) {
  for (int64_t i = 0; i < n_coarse; ++i) ML_TRY(advance(h, h->cfg.num_levels - 1, 1));
  return HLBM_OK;
}

int ml_check_status(hlbm_lattice* h) {
  if (h->d_status == nullptr) return HLBM_OK;
  int st = 0;
  ML_CUDA(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  ML_CUDA(h, cudaStreamSynchronize(h->stream));
  if (st == 1) return fail(h, HLBM_E_BAD_STATE, "a transfer stencil reached a node that is not stored");
  if (st == 2) return fail(h, HLBM_E_BAD_STATE, "rebuild: a new node had no source at any level");
  return HLBM_OK;
}

// Rebuild ---------------------------------------------------------------------

int ml_rebuild(hlbm_lattice* h, const float* pos, int64_t n_pos, int pos_on_device, const int32_t* blocks,
               int64_t n_blocks, int64_t counts_out[3], const std::vector<std::vector<uint8_t>>* H_given) {
  ProfScope prof_scope(h, kProfRebuild);
  const int L = h->cfg.num_levels;
  cudaStream_t st = h->stream;
  const int per[3] = {h->cfg.periodic[0], h->cfg.periodic[1], h->cfg.periodic[2]};
  if (h->d_status == nullptr) {
    ML_TRY(alloc_t(h, &h->d_status, 2));
    ML_CUDA(h, cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st));
  }
  const bool has_old = h->have_blocks && h->device_hierarchy;

  // 1. occupancy of level-0 blocks (Phi = 0 there)
  const GridDims d0 = dims_of(h, 0);
  uint8_t* d_occ = nullptr;
  int* d_bad = h->d_status + 1;
  ML_TRY(alloc_t(h, &d_occ, size_t(d0.slots())));
  std::vector<void*> tmp = {d_occ};
  auto cleanup = [&]() {
    for (void*& p : tmp) LatticeOps::release(h, p);
  };
  ML_CUDA(h, cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  if (H_given != nullptr) {
    // explicit hierarchy: the has-children sets come from the caller
  } else if (blocks != nullptr) {
    int32_t* d_b = nullptr;
    if (n_blocks > 0) {
      if (int rc0 = alloc_t(h, &d_b, size_t(n_blocks) * 3)) {
        cleanup();
        return rc0;
      }
      tmp.push_back(d_b);
      ML_CUDA(h, cudaMemcpyAsync(d_b, blocks, size_t(n_blocks) * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    ML_CUDA(h, occupancy_from_blocks(d_b, n_blocks, d0, d_occ, d_bad, st));
  } else {
    const float* d_p = pos;
    if (!pos_on_device && n_pos > 0) {
      float* d_copy = nullptr;
      if (int rc0 = alloc_t(h, &d_copy, size_t(n_pos) * 3)) {
        cleanup();
        return rc0;
      }
      tmp.push_back(d_copy);
      ML_CUDA(h, cudaMemcpyAsync(d_copy, pos, size_t(n_pos) * 3 * sizeof(float), cudaMemcpyHostToDevice, st));
      d_p = d_copy;
    }
    ML_CUDA(h, occupancy_from_particles(d_p, n_pos, d0, d_occ, d_bad, st));
  }

  // The level-0 occupancy of this call becomes the reference of the next
  // one (particle and block-list rebuilds; an explicit hierarchy has none).
  auto adopt_occupancy = [&]() {
    void* v = h->d_prev_occ;
    LatticeOps::release(h, v);
    h->d_prev_occ = nullptr;
    if (H_given == nullptr) {
      h->d_prev_occ = d_occ;
      tmp[0] = nullptr;  // d_occ: kept, not released with the temporaries
    }
  };

  // The same hierarchy as the installed one: the installed levels stay
  // (lists, neighbour and interface tables, moments); what the full path
  // does to surviving blocks is done in place: the interface refill from the
  // coarser level and the scale refit, and the list flags keep their leaf /
  // border bits only.
  auto keep_installed = [&]() -> int {
    adopt_occupancy();
    cleanup();
    int rc1 = HLBM_OK;
    for (int l = L - 2; l >= 0 && rc1 == HLBM_OK; --l) rc1 = downward(h, l, 1, true);
    for (int l = 0; l < L && rc1 == HLBM_OK; ++l) {
      LevelData& X = h->lv[l];
      if (X.d_list_flags != nullptr) ML_CUDA(h, clear_change_flags(X.d_list_flags, X.nb, st));
      X.host_lists = false;
      rc1 = LatticeOps::maybe_rescale(h, X, true);
    }
    if (rc1) return rc1;
    int status[2] = {0, 0};
    ML_CUDA(h, cudaMemcpyAsync(status, h->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    ML_CUDA(h, cudaStreamSynchronize(st));
    void* v = h->d_F;
    LatticeOps::release(h, v);
    h->d_F = nullptr;
    v = h->d_eps;
    LatticeOps::release(h, v);
    h->d_eps = nullptr;
    ++h->hier_gen;
    if (counts_out != nullptr) counts_out[0] = counts_out[1] = counts_out[2] = 0;
    if (status[0] == 1) return fail(h, HLBM_E_BAD_STATE, "a transfer stencil reached a node that is not stored");
    if (status[1]) return fail(h, HLBM_E_NONFINITE, "%d particle positions are not finite (ignored)", status[1]);
    return HLBM_OK;
  };

  // The hierarchy derives from the level-0 occupancy alone: the occupancy of
  // the installed hierarchy again means the same hierarchy, found before any
  // set or table is built.
  if (has_old && H_given == nullptr && h->d_prev_occ != nullptr) {
    unsigned long long* d_diff = nullptr;
    if (int rc0 = alloc_t(h, &d_diff, 1)) {
      cleanup();
      return rc0;
    }
    tmp.push_back(d_diff);
    unsigned long long diff = 1;
    ML_CUDA(h, cudaMemsetAsync(d_diff, 0, sizeof(unsigned long long), st));
    ML_CUDA(h, count_diff(d_occ, h->d_prev_occ, d0.slots(), d_diff, st));
    ML_CUDA(h, cudaMemcpyAsync(&diff, d_diff, sizeof(diff), cudaMemcpyDeviceToHost, st));
    ML_CUDA(h, cudaStreamSynchronize(st));
    if (diff == 0) return keep_installed();
  }

  // 2. H, I, stored, flags on the dense slot grids
  std::vector<LevelData> nl(L);
  for (int l = 0; l < L; ++l) nl[l].tau = h->lv[l].tau;
  auto free_new = [&]() {
    for (auto& X : nl) LatticeOps::free_level(h, X);
  };
  int rc = HLBM_OK;
  std::vector<uint8_t*> d_I(L, nullptr), d_fl(L, nullptr);
  for (int l = 0; l < L && rc == HLBM_OK; ++l) {
    const size_t ns = size_t(dims_of(h, l).slots());
    if ((rc = alloc_t(h, &nl[l].d_H, ns))) break;
    if ((rc = alloc_t(h, &nl[l].d_stored, ns))) break;
    if ((rc = alloc_t(h, &d_I[l], ns))) break;
    tmp.push_back(d_I[l]);
    if ((rc = alloc_t(h, &d_fl[l], ns))) break;
    tmp.push_back(d_fl[l]);
  }
  if (rc) {
    free_new();
    cleanup();
    return rc;
  }
  ML_CUDA(h, cudaMemsetAsync(nl[0].d_H, 0, size_t(d0.slots()), st));
  for (int l = 1; l < L; ++l) {
    if (H_given != nullptr)
      ML_CUDA(h, cudaMemcpyAsync(nl[l].d_H, (*H_given)[l].data(), size_t(dims_of(h, l).slots()),
                                 cudaMemcpyHostToDevice, st));
    else
      ML_CUDA(h,
              dilate_parent(l == 1 ? d_occ : nl[l - 1].d_H, dims_of(h, l - 1), nl[l].d_H, dims_of(h, l), per, st));
  }
  for (int l = 0; l < L; ++l)
    ML_CUDA(h, internal_stored(nl[l].d_H, l < L - 1 ? nl[l + 1].d_H : nullptr, dims_of(h, l),
                               l < L - 1 ? dims_of(h, l + 1) : dims_of(h, l), per, l >= 1, d_I[l], nl[l].d_stored,
                               st));
  for (int l = 0; l < L; ++l)
    ML_CUDA(h, slot_flags(nl[l].d_stored, nl[l].d_H, l < L - 1 ? nl[l + 1].d_stored : nullptr, dims_of(h, l),
                          l < L - 1 ? dims_of(h, l + 1) : dims_of(h, l), has_old ? h->lv[l].d_stored : nullptr,
                          has_old ? h->lv[l].d_H : nullptr, has_old, d_fl[l], st));

  // 3. stable compaction of every level
  int64_t* d_cnt = nullptr;
  int64_t max_cta = 0;
  for (int l = 0; l < L; ++l) max_cta = std::max<int64_t>(max_cta, (dims_of(h, l).slots() + 1023) / 1024);
  if ((rc = alloc_t(h, &d_cnt, size_t(max_cta) + 4 * L + 8))) {
    free_new();
    cleanup();
    return rc;
  }
  tmp.push_back(d_cnt);
  int64_t* d_tot = d_cnt + max_cta;  // [L] block counts, then [2L] interface counts
  std::vector<uint8_t*> d_lflags(L, nullptr);
  for (int l = 0; l < L && rc == HLBM_OK; ++l) {
    const size_t ns = size_t(dims_of(h, l).slots());
    if ((rc = alloc_t(h, &nl[l].d_slot, ns))) break;
    if ((rc = alloc_t(h, &nl[l].d_coords, ns * 3))) break;
    if ((rc = alloc_t(h, &nl[l].d_skip, ns))) break;
    if ((rc = alloc_t(h, &d_lflags[l], ns))) break;
    nl[l].d_list_flags = d_lflags[l];
    cudaError_t e = compact_slots(nl[l].d_stored, d_fl[l], nl[l].d_H, dims_of(h, l), nl[l].d_slot, nl[l].d_coords,
                                  d_lflags[l], nl[l].d_skip, d_cnt, d_tot + l, st);
    if (e != cudaSuccess) rc = fail(h, HLBM_E_CUDA, "compaction: %s", cudaGetErrorString(e));
  }
  if (rc) {
    free_new();
    cleanup();
    return rc;
  }
  // changes against the installed hierarchy, read back with the block counts
  unsigned long long changes[4] = {0, 0, 0, 0};
  unsigned long long* d_changes = reinterpret_cast<unsigned long long*>(d_tot + 3 * L);
  if (has_old) {
    ML_CUDA(h, cudaMemsetAsync(d_changes, 0, 4 * sizeof(unsigned long long), st));
    for (int l = 0; l < L; ++l)
      ML_CUDA(h, count_changes(nl[l].d_H, h->lv[l].d_H, nl[l].d_stored, h->lv[l].d_stored, dims_of(h, l).slots(),
                               d_changes, st));
    ML_CUDA(h, cudaMemcpyAsync(changes, d_changes, sizeof(changes), cudaMemcpyDeviceToHost, st));
  }
  std::vector<int64_t> nb(L);
  ML_CUDA(h, cudaMemcpyAsync(nb.data(), d_tot, L * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  ML_CUDA(h, cudaStreamSynchronize(st));
  if (has_old && changes[0] == 0 && changes[1] == 0 && changes[2] == 0 && changes[3] == 0) {
    free_new();
    return keep_installed();
  }

  // 4. neighbour tables and interface node lists; with the spatial-hash block
  // table, each level's hash is built from its list first, the neighbour
  // table is found through it, and the dense slot table is dropped
  for (int l = 0; l < L && rc == HLBM_OK; ++l) {
    nl[l].nb = nb[l];
    if (nb[l] == 0) continue;
    if ((rc = alloc_t(h, &nl[l].d_nbr, size_t(nb[l]) * 27))) break;
    const int32_t* slot = nl[l].d_slot;
    BlockHash hash{};
    if (h->block_lookup == 1) {
      nl[l].hcap = hash_capacity(nb[l]);
      if ((rc = alloc_t(h, &nl[l].d_hkeys, nl[l].hcap))) break;
      if ((rc = alloc_t(h, &nl[l].d_hvals, nl[l].hcap))) break;
      cudaError_t e = build_block_hash(nl[l].d_coords, nb[l], nl[l].d_hkeys, nl[l].d_hvals, nl[l].hcap, st);
      if (e != cudaSuccess) {
        rc = fail(h, HLBM_E_CUDA, "block hash: %s", cudaGetErrorString(e));
        break;
      }
      hash = BlockHash{nl[l].d_hkeys, nl[l].d_hvals, nl[l].hcap - 1u};
      slot = nullptr;
    }
    cudaError_t e = neighbour_table(nl[l].d_coords, nb[l], slot, dims_of(h, l), per, h->open_mask(), nl[l].d_nbr, st,
                                    hash);
    if (e != cudaSuccess) rc = fail(h, HLBM_E_CUDA, "neighbour table: %s", cudaGetErrorString(e));
    if (rc == HLBM_OK) rc = LatticeOps::bounce(h, nl[l]);
  }
  std::vector<int64_t*> d_ioff(L, nullptr);
  for (int l = 0; l < L && rc == HLBM_OK; ++l) {
    if (nb[l] == 0) continue;
    if ((rc = alloc_t(h, &d_ioff[l], size_t(nb[l]) * 2 + 2))) break;
    tmp.push_back(d_ioff[l]);
    cudaError_t e = interface_count(nl[l].d_nbr, nl[l].d_skip, nb[l], d_ioff[l], d_tot + L + 2 * l, st);
    if (e != cudaSuccess) rc = fail(h, HLBM_E_CUDA, "interface count: %s", cudaGetErrorString(e));
  }
  if (rc) {
    free_new();
    cleanup();
    return rc;
  }
  std::vector<int64_t> ic(2 * L, 0);
  for (int l = 0; l < L; ++l)
    if (nb[l] == 0) ML_CUDA(h, cudaMemsetAsync(d_tot + L + 2 * l, 0, 2 * sizeof(int64_t), st));
  ML_CUDA(h, cudaMemcpyAsync(ic.data(), d_tot + L, 2 * L * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  ML_CUDA(h, cudaStreamSynchronize(st));
  for (int l = 0; l < L && rc == HLBM_OK; ++l) {
    nl[l].n_down = ic[2 * l];
    nl[l].n_up = ic[2 * l + 1];
    if (nb[l] == 0) continue;
    if ((rc = alloc_t(h, &nl[l].d_down, size_t(nl[l].n_down) + 1))) break;
    if ((rc = alloc_t(h, &nl[l].d_up, size_t(nl[l].n_up) + 1))) break;
    if (l + 1 < L && (rc = alloc_t(h, &nl[l].d_down_acc, size_t(nl[l].n_down) * 10 + 1))) break;
    if (l + 1 < L && (rc = alloc_t(h, &nl[l].d_down_t, size_t(nl[l].n_down) + 1))) break;
    if (l + 1 < L && (rc = alloc_t(h, &nl[l].d_down_stc, size_t(nl[l].n_down) * 8 + 1))) break;
    cudaError_t e = interface_scatter(nl[l].d_nbr, nl[l].d_skip, nb[l], d_ioff[l], nl[l].d_down, nl[l].d_up, st);
    if (e != cudaSuccess) {
      rc = fail(h, HLBM_E_CUDA, "interface scatter: %s", cudaGetErrorString(e));
      break;
    }
    if (l + 1 < L && nl[l].n_down > 0) {
      int64_t* d_ord = nullptr;
      if ((rc = alloc_t(h, &d_ord, size_t(transfer_order_scratch(nl[l].n_down))))) break;
      tmp.push_back(d_ord);
      e = transfer_order(nl[l].d_down, nl[l].n_down, d_ord, nl[l].d_down_t, st);
      if (e == cudaSuccess) {
        TransferArgs t{};
        t.fine = view_of(nl[l], dims_of(h, l));
        t.coarse = view_of(nl[l + 1], dims_of(h, l + 1));
        t.nodes = nl[l].d_down_t;
        t.n_nodes = nl[l].n_down;
        for (int ax = 0; ax < 3; ++ax) t.periodic[ax] = h->cfg.periodic[ax];
        t.status = h->d_status;
        e = down_stencil(t, nl[l].d_down_stc, st);
      }
      if (e != cudaSuccess) rc = fail(h, HLBM_E_CUDA, "transfer order: %s", cudaGetErrorString(e));
    }
  }

  // 5. moments: survivors keep theirs, new nodes take the transfer rules
  const size_t node_bytes = kRows * storage_size(h->cfg.storage);
  for (int l = 0; l < L && rc == HLBM_OK; ++l)
    for (int k = 0; k < 2 && rc == HLBM_OK; ++k)
      rc = LatticeOps::alloc(h, &nl[l].d_mom[k], size_t(nb[l]) * kCells * node_bytes);
  if (rc) {
    free_new();
    cleanup();
    return rc;
  }
  for (int l = 0; l < L && rc == HLBM_OK; ++l) {
    rc = LatticeOps::init_scales(h, nl[l]);
    // moments carried over from every old level: start from the widest range
    // of the old level and refit below
    if (rc == HLBM_OK && has_old && nl[l].d_scales != nullptr && h->lv[l].d_scales != nullptr)
      ML_CUDA(h, cudaMemcpyAsync(nl[l].d_scales, h->lv[l].d_scales, sizeof(Scales), cudaMemcpyDeviceToDevice, st));
  }
  // every old level at the same time: refill I^d from the coarser level, so
  // that new nodes interpolate from a current interface.  This is the first
  // write to the old state and comes after the last allocation, so a rebuild
  // that fails for memory leaves the old hierarchy as it was.
  if (rc == HLBM_OK && has_old)
    for (int l = L - 2; l >= 0 && rc == HLBM_OK; --l) rc = downward(h, l, 1, true);
  if (rc) {
    free_new();
    cleanup();
    return rc;
  }
  if (has_old) {
    OldHierarchy o{};
    o.L = L;
    for (int l = 0; l < L; ++l) {
      o.lv[l] = view_of(h->lv[l], dims_of(h, l));
      o.kup[l] = h->kup[l];
      o.kdown[l] = h->kdown[l];
    }
    for (int ax = 0; ax < 3; ++ax) o.periodic[ax] = per[ax];
    o.ext[0] = h->cfg.nx;
    o.ext[1] = h->cfg.ny;
    o.ext[2] = h->cfg.nz;
    for (int l = 0; l < L; ++l)
      ML_CUDA(h, init_new_level(h->cfg.storage, o, l, nl[l].d_coords, nb[l], nl[l].d_mom[0], nl[l].d_scales,
                                h->d_status, st));
  } else {
    for (int l = 0; l < L; ++l)
      if (nb[l]) ML_CUDA(h, cudaMemsetAsync(nl[l].d_mom[0], 0, size_t(nb[l]) * kCells * node_bytes, st));
  }
  // only the current buffer needs the state: every level steps (writing the
  // other buffer) before anything reads its previous state
  for (int l = 0; l < L; ++l) {
    nl[l].cur = 0;
    ML_TRY(LatticeOps::maybe_rescale(h, nl[l], true));
  }

  // 6. the counts of refined / coarsened / deleted blocks came back with the
  // block counts
  // the host copies of the block lists are made on demand (hlbm_get_blocks);
  // one readback brings the status words (transfer status, dropped particles)
  for (int l = 0; l < L; ++l) nl[l].host_lists = false;
  int status[2] = {0, 0};
  ML_CUDA(h, cudaMemcpyAsync(status, h->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  ML_CUDA(h, cudaStreamSynchronize(st));
  const int64_t refined = int64_t(changes[0]), coarsened = int64_t(changes[1]), deleted = int64_t(changes[2]);
  const int bad = status[1];
  adopt_occupancy();
  cleanup();
  for (auto& X : h->lv) LatticeOps::free_level(h, X);
  for (int l = 0; l < L; ++l) {
    nl[l].cur = 0;
    if (h->block_lookup == 1 && nl[l].d_hkeys != nullptr) {  // the hash replaces the slot table
      void* v = nl[l].d_slot;
      LatticeOps::release(h, v);
      nl[l].d_slot = nullptr;
    }
    h->lv[l] = nl[l];
  }
  // the level-0 force field refers to the old block list
  void* v = h->d_F;
  LatticeOps::release(h, v);
  h->d_F = nullptr;
  v = h->d_eps;
  LatticeOps::release(h, v);
  h->d_eps = nullptr;
  h->have_blocks = true;
  h->device_hierarchy = true;
  ++h->hier_gen;
  if (counts_out != nullptr) {
    counts_out[0] = refined;
    counts_out[1] = coarsened;
    counts_out[2] = deleted;
  }
  if (status[0] == 1) return fail(h, HLBM_E_BAD_STATE, "a transfer stencil reached a node that is not stored");
  if (status[0] == 2) return fail(h, HLBM_E_BAD_STATE, "rebuild: a new node had no source at any level");
  if (bad) return fail(h, HLBM_E_NONFINITE, "%d particle positions are not finite (ignored)", bad);
  return HLBM_OK;
}

// Explicit hierarchies (hlbm_set_blocks) -----------------------------------------

namespace {

// A dense per-level block grid on the host, indexed like the slot tables.
struct HostGrid {
  GridDims d;
  std::vector<uint8_t> v;
  explicit HostGrid(GridDims dd) : d(dd), v(size_t(dd.slots()), 0) {}
  uint8_t& at(int x, int y, int z) { return v[(size_t(z) * d.ny + y) * d.nx + x]; }
  uint8_t at(int x, int y, int z) const { return v[(size_t(z) * d.ny + y) * d.nx + x]; }
};

// Value of G at (x+dx, y+dy, z+dz): wrapped on periodic axes, `fill` beyond a wall.
uint8_t nbr_of(const HostGrid& G, int x, int y, int z, int dx, int dy, int dz, const int per[3], uint8_t fill) {
  int c[3] = {x + dx, y + dy, z + dz};
  const int n[3] = {G.d.nx, G.d.ny, G.d.nz};
  for (int a = 0; a < 3; ++a) {
    if (c[a] >= 0 && c[a] < n[a]) continue;
    if (!per[a]) return fill;
    c[a] = (c[a] % n[a] + n[a]) % n[a];
  }
  return G.at(c[0], c[1], c[2]);
}

// One-block dilation in the 26-neighbourhood (clipped at walls) or erosion
// (a block whose every in-domain neighbour is set: the internal blocks).
HostGrid morph(const HostGrid& G, const int per[3], bool erode) {
  HostGrid out(G.d);
  for (int z = 0; z < G.d.nz; ++z)
    for (int y = 0; y < G.d.ny; ++y)
      for (int x = 0; x < G.d.nx; ++x) {
        uint8_t r = G.at(x, y, z);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const uint8_t q = nbr_of(G, x, y, z, dx, dy, dz, per, erode ? 1 : 0);
              r = erode ? uint8_t(r & q) : uint8_t(r | q);
            }
        out.at(x, y, z) = r;
      }
  return out;
}

// Level-(l+1) grid: a block is set if any of its 2x2x2 children is set.
HostGrid parent_of(const HostGrid& G, GridDims du) {
  HostGrid out(du);
  for (int z = 0; z < G.d.nz; ++z)
    for (int y = 0; y < G.d.ny; ++y)
      for (int x = 0; x < G.d.nx; ++x)
        if (G.at(x, y, z)) out.at(x >> 1, y >> 1, z >> 1) = 1;
  return out;
}

}  // namespace

int ml_set_blocks(hlbm_lattice* h, int level, const int32_t* coords, int64_t n) {
  const int L = h->cfg.num_levels;
  if (int(h->staged.size()) != L) {
    h->staged.assign(size_t(L), 0);
    h->staged_blocks.assign(size_t(L), {});
  }
  const GridDims d = dims_of(h, level);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* c = coords + 3 * i;
    if (c[0] < 0 || c[0] >= d.nx || c[1] < 0 || c[1] >= d.ny || c[2] < 0 || c[2] >= d.nz)
      return fail(h, HLBM_E_INVALID_ARG, "level %d block %lld (%d, %d, %d) is outside the %d x %d x %d block grid",
                  level, (long long)i, c[0], c[1], c[2], d.nx, d.ny, d.nz);
  }
  h->staged_blocks[size_t(level)].assign(coords, coords + 3 * n);
  h->staged[size_t(level)] = 1;
  for (int l = 0; l < L; ++l)
    if (!h->staged[size_t(l)]) return HLBM_OK;  // wait for the other levels

  // every level staged: validate and install.  The staged lists are consumed
  // either way.
  std::vector<std::vector<int32_t>> lists;
  lists.swap(h->staged_blocks);
  h->staged.assign(size_t(L), 0);
  h->staged_blocks.assign(size_t(L), {});
  const int per[3] = {h->cfg.periodic[0], h->cfg.periodic[1], h->cfg.periodic[2]};
  std::vector<HostGrid> S, H, I;
  for (int l = 0; l < L; ++l) {
    S.emplace_back(dims_of(h, l));
    const std::vector<int32_t>& c = lists[size_t(l)];
    for (size_t i = 0; i < c.size() / 3; ++i) {
      uint8_t& cell = S[size_t(l)].at(c[3 * i], c[3 * i + 1], c[3 * i + 2]);
      if (cell)
        return fail(h, HLBM_E_INVALID_ARG, "level %d block (%d, %d, %d) is listed twice", l, c[3 * i],
                    c[3 * i + 1], c[3 * i + 2]);
      cell = 1;
    }
  }
  // bottom-up: H_l = blocks with stored or internal children, I_l = H_l blocks
  // whose every in-domain neighbour is in H_l (covered, not stored)
  H.emplace_back(dims_of(h, 0));
  I.emplace_back(dims_of(h, 0));
  for (int l = 1; l < L; ++l) {
    HostGrid R = S[size_t(l - 1)];
    for (size_t q = 0; q < R.v.size(); ++q) R.v[q] |= I[size_t(l - 1)].v[q];
    H.push_back(parent_of(R, dims_of(h, l)));
    I.push_back(morph(H.back(), per, true));
    for (size_t q = 0; q < H.back().v.size(); ++q) I.back().v[q] &= H.back().v[q];
  }
  for (int l = 0; l < L; ++l) {
    const GridDims dl = dims_of(h, l);
    for (int z = 0; z < dl.nz; ++z)
      for (int y = 0; y < dl.ny; ++y)
        for (int x = 0; x < dl.nx; ++x) {
          const bool st = S[size_t(l)].at(x, y, z) != 0, in = I[size_t(l)].at(x, y, z) != 0;
          if (st && in)
            return fail(h, HLBM_E_INVALID_ARG,
                        "level %d block (%d, %d, %d) is stored but internal: it and its 26 neighbours all have "
                        "finer children (Sec. 6.1 stores leaf and border blocks only)",
                        l, x, y, z);
          if (l + 1 < L) {
            const bool pst = S[size_t(l + 1)].at(x >> 1, y >> 1, z >> 1) != 0;
            const bool pin = I[size_t(l + 1)].at(x >> 1, y >> 1, z >> 1) != 0;
            const bool refined = H[size_t(l + 1)].at(x >> 1, y >> 1, z >> 1) != 0;
            if (st && !pst && !pin)
              return fail(h, HLBM_E_INVALID_ARG,
                          "level %d block (%d, %d, %d) has a parent that is neither stored nor internal at level %d",
                          l, x, y, z, l + 1);
            if (refined && !in && !st)
              return fail(h, HLBM_E_INVALID_ARG,
                          "level %d block (%d, %d, %d) is missing: its parent at level %d has other children, so "
                          "all 8 must be stored or internal",
                          l, x, y, z, l + 1);
          } else if (!st && !in) {
            return fail(h, HLBM_E_INVALID_ARG,
                        "top level %d block (%d, %d, %d) is missing: the top level covers every block that is not "
                        "internal",
                        l, x, y, z);
          }
        }
  }
  // overlap and separation: every refined set is a union of 3x3x3-block
  // cubes (each refined block lies within one block of a block whose whole
  // neighbourhood is refined), so a finer region keeps one coarse block of
  // overlap with the coarser level; and a region refined at level l - 1 is
  // surrounded by one level-(l+1) block of level-l blocks (2:1 grading: two
  // levels apart never touch)
  for (int l = 1; l < L; ++l) {
    const HostGrid open = morph(I[size_t(l)], per, false);
    for (size_t q = 0; q < open.v.size(); ++q)
      if (open.v[q] != H[size_t(l)].v[q])
        return fail(h, HLBM_E_INVALID_ARG,
                    "level %d: the region refined below level %d is not a union of 3x3x3-block cubes at slot %lld "
                    "(the finer level needs one level-%d block of overlap around it)",
                    l - 1, l, (long long)q, l);
    if (l + 1 < L) {
      const HostGrid need = morph(parent_of(H[size_t(l)], dims_of(h, l + 1)), per, false);
      for (size_t q = 0; q < need.v.size(); ++q)
        if (need.v[q] && !H[size_t(l + 1)].v[q])
          return fail(h, HLBM_E_INVALID_ARG,
                      "level %d slot %lld: a block next to the level-%d region is not refined (2:1 grading needs "
                      "one level-%d block of level-%d cells around every level-%d region)",
                      l + 1, (long long)q, l - 1, l + 1, l, l - 1);
    }
  }
  std::vector<std::vector<uint8_t>> Hv(static_cast<size_t>(L));
  for (int l = 0; l < L; ++l) Hv[size_t(l)] = H[size_t(l)].v;
  return ml_rebuild(h, nullptr, 0, 0, nullptr, 0, nullptr, &Hv);
}

}  // namespace hlbm
