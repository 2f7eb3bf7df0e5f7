// adjoint_ml.cu -- reverse mode of the multi-level advance (Algorithm 1) with
// FP32 storage: the transposed downward and upward transfers (Sec. 5.2 and
// 5.3, with their S^neq rescaling) and the checkpointed driver behind
// hlbm_forward_record / hlbm_adjoint for lattices with a device hierarchy.
//
// One coarse step of Algorithm 1 is a fixed sequence of operations on the
// per-level states A_l (read buffer) and P_l (the state before the level's
// last step, read by the downward transfer of the next finer level):
//   SC(l)      P_l <- A_l, A_l <- step(A_l)          (interface nodes copy)
//   DOWN(l, s) A_l[I^d_l] <- D(P_{l+1}) (s = 1) or D((P_{l+1} + A_{l+1}) / 2)
//   UP(l)      A_{l+1}[I^u_{l+1}] <- U(A_l)
// The reverse pass walks that sequence backwards with the adjoints lambda_A,
// lambda_P of every level:
//   SC^T    lambda_A <- (d step / d A)^T lambda_A + lambda_P, lambda_P <- 0
//   DOWN^T  lambda_P_{l+1} (and lambda_A_{l+1} at s = 2) += (dD)^T lambda_A_l[I^d],
//           lambda_A_l[I^d] <- 0
//   UP^T    lambda_A_l += (dU)^T lambda_A_{l+1}[I^u], lambda_A_{l+1}[I^u] <- 0
// Each checkpoint segment is recomputed first: every SC writes a fresh output
// buffer and its pre-collision moments; the transfers write in place and keep
// the values they overwrite (an undo log), which the reverse pass puts back,
// so that every operation sees its inputs as they were in the forward run.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "adjoint_math.cuh"
#include "f2_common.cuh"
#include "fp64_bits.cuh"
#include "hierarchy.cuh"
#include "hlbm_internal.h"
#include "lattice_state.h"
#include "multilevel.cuh"

namespace hlbm {
namespace {

constexpr int64_t kBlockVals = int64_t(kRows) * kCells;

__device__ __forceinline__ int64_t find_block(const LevelView& v, int x, int y, int z) {
  const int bx = x >> 3, by = y >> 3, bz = z >> 3;
  if (bx < 0 || by < 0 || bz < 0 || bx >= v.d.nx || by >= v.d.ny || bz >= v.d.nz) return -1;
  if (v.hash.keys != nullptr) return hash_find(v.hash, bx, by, bz);
  return v.slot[(int64_t(bz) * v.d.ny + by) * v.d.nx + bx];
}

__device__ __forceinline__ int node_cell(int x, int y, int z) { return (x & 7) + 8 * (y & 7) + 64 * (z & 7); }

// Coarse stencil indices along one axis, as the downward transfer takes them.
__device__ __forceinline__ void stencil_axis(int p, int n, int periodic, int& lo, int& hi) {
  lo = p >> 1;
  hi = (p + 1) >> 1;
  if (hi >= n) hi = periodic ? hi - n : n - 1;
}

// Moments (delta_rho, u, S) of a node of an FP32 level (paired node order).
__device__ __forceinline__ void load_f32(const void* base, int64_t blk, int cell, float (&m)[kRows]) {
  const float* p = static_cast<const float*>(base) + blk * kBlockVals + node_offset<float>(cell);
#pragma unroll
  for (int r = 0; r < kRows; ++r) m[r] = p[r * kCells];
}

// The adjoint, with respect to stored moments m (delta_rho, u, S), of a
// weighted S^neq = S - u u split: lam_rho, lam_u (before the split) and
// lam_sn, all times w.
__device__ __forceinline__ void split_adjoint(const float (&m)[kRows], float w, float lrho, const float (&lu)[3],
                                              const float (&lsn)[6], float (&v)[kRows]) {
  const float ux = m[1], uy = m[2], uz = m[3];
  v[0] = w * lrho;
  v[1] = w * (lu[0] - (2.f * ux * lsn[0] + uy * lsn[3] + uz * lsn[4]));
  v[2] = w * (lu[1] - (2.f * uy * lsn[1] + ux * lsn[3] + uz * lsn[5]));
  v[3] = w * (lu[2] - (2.f * uz * lsn[2] + ux * lsn[4] + uy * lsn[5]));
#pragma unroll
  for (int r = 0; r < 6; ++r) v[4 + r] = w * lsn[r];
}

__device__ __forceinline__ void add10(float* lam, const float (&v)[kRows]) {
#pragma unroll
  for (int r = 0; r < kRows; ++r) lam[r * kCells] += v[r];
}

// Pass-through nodes of a level: solid nodes and nodes next to a neighbour
// block that is not stored (interface nodes), which copy their input in the
// forward step.  Bit (cell & 31) of word [blk][cell >> 5], natural order.
__global__ void __launch_bounds__(kCells) k_passthrough_bits(const int32_t* __restrict__ nbr,
                                                             const uint8_t* __restrict__ bflags,
                                                             const uint8_t* __restrict__ solid,
                                                             uint32_t* __restrict__ bits) {
  __shared__ unsigned s_miss;
  const int64_t blk = blockIdx.x;
  const int t = threadIdx.x;
  if (t < 32) {
    const int v = t < 27 ? nbr[blk * 27 + t] : 0;
    const unsigned mb = __ballot_sync(0xffffffffu, t < 27 && is_copy_nbr(v));
    if (t == 0) s_miss = mb;
  }
  __syncthreads();
  bool p = s_miss != 0u && f2::touches_missing(t & 7, (t >> 3) & 7, t >> 6, s_miss);
  if (bflags != nullptr && (bflags[blk] & kBlockSolidNear)) p = p || solid[blk * kCells + t] != 0;
  const unsigned b = __ballot_sync(0xffffffffu, p);
  if ((t & 31) == 0) bits[blk * (kCells / 32) + (t >> 5)] = b;
}

// Where an addition to a level's lambda goes.  A plain level (pt null) holds
// lambda in raw.  A fused level holds, after the reverse stream of its last
// reversed step (which applied the transposed collision of the step before
// it), mu = lambda_p of that earlier step at ordinary nodes (zero at
// pass-through nodes) and lambda itself at pass-through nodes, in raw.  An
// addition dlam at an ordinary node of a fused level goes through that
// transposed collision (recorded p = pre): (dC/dp)^T dlam into mu and, on the
// level with the force field, (dC/dF)^T dlam into dL/dF; the map is linear in
// dlam, so additions may come one by one.  Each node has one writer per
// launch (no atomics).
struct LamTarget {
  const uint32_t* pt;  // pass-through bits, or null (plain)
  float* raw;
  float* mu;
  const float* pre;
  const float* F;      // force field [nb][3][512] or null (uniform fu)
  const float* eps;    // fluid fraction [nb][512] or null
  float fu[3];
  float om, tau;
  float* dF;           // dL/dF of the current checkpoint segment [nb][3][512] (FP32), or null
};

__device__ __forceinline__ void add_lambda(const LamTarget& g, int64_t blk, int cell, const float (&v)[kRows]) {
  const int64_t o = blk * kBlockVals + cell;
  if (g.pt == nullptr || ((g.pt[blk * (kCells / 32) + (cell >> 5)] >> (cell & 31)) & 1u)) {
    add10(g.raw + o, v);
    return;
  }
  const float* q = g.pre + o;
  PreMom<float> p;
  p.drho = q[0];
  p.jx = q[kCells];
  p.jy = q[2 * kCells];
  p.jz = q[3 * kCells];
  p.pxx = q[4 * kCells];
  p.pyy = q[5 * kCells];
  p.pzz = q[6 * kCells];
  p.pxy = q[7 * kCells];
  p.pxz = q[8 * kCells];
  p.pyz = q[9 * kCells];
  float fx = g.fu[0], fy = g.fu[1], fz = g.fu[2];
  if (g.F != nullptr) {
    const float* f = g.F + blk * 3 * kCells + cell;
    fx = f[0];
    fy = f[kCells];
    fz = f[2 * kCells];
  }
  const float om = g.eps != nullptr ? 1.f / (g.tau * g.eps[blk * kCells + cell]) : g.om;
  Mom<float> lo;
  lo.drho = v[0];
  lo.ux = v[1];
  lo.uy = v[2];
  lo.uz = v[3];
  lo.sxx = v[4];
  lo.syy = v[5];
  lo.szz = v[6];
  lo.sxy = v[7];
  lo.sxz = v[8];
  lo.syz = v[9];
  PreMom<float> lp;
  float lfx, lfy, lfz;
  collide_vjp(p, fx, fy, fz, om, lo, lp, lfx, lfy, lfz);
  const float w[kRows] = {lp.drho, lp.jx, lp.jy, lp.jz, lp.pxx, lp.pyy, lp.pzz, lp.pxy, lp.pxz, lp.pyz};
  add10(g.mu + o, w);
  if (g.dF != nullptr) {
    float* d = g.dF + blk * 3 * kCells + cell;
    d[0] += lfx;
    d[kCells] += lfy;
    d[2 * kCells] += lfz;
  }
}

struct DownAdjArgs {
  LevelView fine, coarse;  // coarse.mom = A_{l+1} (new), coarse.mom_other = P_{l+1} (old)
  const int32_t* nodes;    // I^d_l: (block << 9) | cell
  const int32_t* stencil;  // seeds: the forward transfer's stencil table, in the order of nodes
  int64_t n_nodes;
  int avg;                 // 1: s = 2 (temporal midpoint), 0: s = 1 (old state only)
  float k;                 // S^neq factor of the transfer
  int periodic[3];
  float* lam_fine;         // lambda_A_l at pass-through nodes, natural order: read at I^d, then zeroed
  LamTarget lam_new;       // lambda_A_{l+1} (s = 2)
  float* lam_old;          // lambda_P_{l+1}
};

// Transposed downward transfer.  The forward value at fine node n is
//   rho = sum_j w_j rho_j, u = sum_j w_j u_j, sn = sum_j w_j (S_j - u_j u_j),
//   stored (rho - 1, u, k sn + u u)
// over the distinct coarse stencil nodes j (and over the old and new states
// with weight 1/2 each at s = 2).  With lam = dL/d(stored) at n, the adjoint
// with respect to (rho, u, sn) at n is the seed
//   (lam_rho, lam_u + (d(u u)/du)^T lam_S, k lam_S),
// and coarse node j receives, for every fine node n whose stencil holds it,
// w_j times the transposed split S^neq = S - u_j u_j of the seed, taken at
// j's own moments.  That map is linear in the seed, so j sums the weighted
// seeds of its fine nodes first and applies it once: two passes, no atomics.

// Pass 1, per I^d node: its seed, written over its lambda (which ends here:
// the transfer overwrote the node).
__global__ void k_down_adj_seed(DownAdjArgs a) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n_nodes) return;
  const int32_t v = a.nodes[k];
  const int64_t b = v >> 9;
  const int cell = v & 511;
  float* lf = a.lam_fine + b * kBlockVals + cell;
  // the stencil from the forward transfer's table (same order as nodes)
  const int nmax = (1 + (cell & 1)) * (1 + ((cell >> 3) & 1)) * (1 + ((cell >> 6) & 1));
  int64_t cb[8];
  int cc[8];
  int nq = 0;
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int32_t st = q < nmax ? a.stencil[q * a.n_nodes + k] : -1;
    nq += st >= 0 ? 1 : 0;
    ok = ok && st != -2;
    cb[q] = st >= 0 ? (st >> 9) : 0;
    cc[q] = st & 511;
  }
  if (!ok) {  // the forward transfer reported this already
#pragma unroll
    for (int r = 0; r < kRows; ++r) lf[r * kCells] = 0.f;
    return;
  }
  // weight 1/nq = 2^-e, halved at s = 2 (old and new state each count half)
  const int e = (nq >= 2 ? 1 : 0) + (nq >= 4 ? 1 : 0) + (nq >= 8 ? 1 : 0) + (a.avg ? 1 : 0);
  const double w = e == 0 ? 1.0 : e == 1 ? 0.5 : e == 2 ? 0.25 : e == 3 ? 0.125 : 0.0625;
  float L[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) L[r] = lf[r * kCells];
  // the interpolated velocity (FP64 sums as in the forward transfer)
  double su[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (q >= nq) break;
    float m[kRows];
    if (a.avg) {
      float o[kRows];
      load_f32(a.coarse.mom_other, cb[q], cc[q], o);
      load_f32(a.coarse.mom, cb[q], cc[q], m);
      for (int ax = 0; ax < 3; ++ax) {
        su[ax] += w * to64(o[1 + ax]);
        su[ax] += w * to64(m[1 + ax]);
      }
    } else {
      load_f32(a.coarse.mom_other, cb[q], cc[q], m);
      for (int ax = 0; ax < 3; ++ax) su[ax] += w * to64(m[1 + ax]);
    }
  }
  const float ux = to32(su[0]), uy = to32(su[1]), uz = to32(su[2]);
  // adjoint of stored S = k sn + u u and of u
  lf[kCells] = L[1] + 2.f * ux * L[4] + uy * L[7] + uz * L[8];
  lf[2 * kCells] = L[2] + 2.f * uy * L[5] + ux * L[7] + uz * L[9];
  lf[3 * kCells] = L[3] + 2.f * uz * L[6] + ux * L[8] + uy * L[9];
#pragma unroll
  for (int r = 4; r < kRows; ++r) lf[r * kCells] = a.k * L[r];
}

// Fine nodes along one axis whose stencil holds coarse index X (n coarse
// nodes, 2n fine): 2X - 1 (wrapped on a periodic axis), 2X, 2X + 1, each
// with its stencil width (1 or 2) along the axis, and whether it exists.
__device__ __forceinline__ void fine_candidates(int X, int n, int periodic, int (&p)[3], int (&wdt)[3],
                                                bool (&ok)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int q = 2 * X + d - 1;
    ok[d] = q >= 0 || periodic;
    if (q < 0) q += 2 * n;
    int lo, hi;
    stencil_axis(q, n, periodic, lo, hi);
    ok[d] = ok[d] && (lo == X || hi == X);
    p[d] = q;
    wdt[d] = lo != hi ? 2 : 1;
  }
}

// Pass 2, per coarse node that some I^d stencil holds: the weighted seeds of
// its fine nodes (bits: the I^d nodes of the fine level), the transposed split
// at its old and, at s = 2, new moments, added to lambda_P and lambda_A.
__global__ void k_down_adj_gather(DownAdjArgs a, const int32_t* __restrict__ targets, int64_t n_targets,
                                  const uint32_t* __restrict__ fine_bits) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_targets) return;
  const int32_t v = targets[t];
  const int64_t cb = v >> 9;
  const int cc = v & 511;
  const int32_t* c = a.coarse.coords + 3 * cb;
  const int X[3] = {c[0] * 8 + (cc & 7), c[1] * 8 + ((cc >> 3) & 7), c[2] * 8 + (cc >> 6)};
  const int n[3] = {a.coarse.d.nx * 8, a.coarse.d.ny * 8, a.coarse.d.nz * 8};
  int px[3], py[3], pz[3], wx[3], wy[3], wz[3];
  bool okx[3], oky[3], okz[3];
  fine_candidates(X[0], n[0], a.periodic[0], px, wx, okx);
  fine_candidates(X[1], n[1], a.periodic[1], py, wy, oky);
  fine_candidates(X[2], n[2], a.periodic[2], pz, wz, okz);
  // The candidates 2X and 2X + 1 of an axis share a block (2X is even); only
  // 2X - 1 may lie in another one.  So the 27 candidates lie in at most 8
  // blocks: look those up first, then test all candidates' I^d bits, then
  // load the seeds of the candidates that hold one (independent loads in
  // each phase).
  int64_t fbk[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int sx = j & 1, sy = (j >> 1) & 1, sz = j >> 2;  // 0: the block of 2X - 1, 1: of 2X
    const bool need = (sx || okx[0]) && (sy || oky[0]) && (sz || okz[0]);
    fbk[j] = need ? find_block(a.fine, px[sx ? 1 : 0], py[sy ? 1 : 0], pz[sz ? 1 : 0]) : -1;
  }
  uint32_t hit = 0;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int ix = q % 3, iy = (q / 3) % 3, iz = q / 9;
    const int64_t fb = fbk[(ix ? 1 : 0) | (iy ? 2 : 0) | (iz ? 4 : 0)];
    if (!(okx[ix] && oky[iy] && okz[iz]) || fb < 0) continue;
    const int fc = node_cell(px[ix], py[iy], pz[iz]);
    if ((__ldg(fine_bits + fb * (kCells / 32) + (fc >> 5)) >> (fc & 31)) & 1u) hit |= 1u << q;
  }
  float acc[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) acc[r] = 0.f;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (!((hit >> q) & 1u)) continue;
    const int ix = q % 3, iy = (q / 3) % 3, iz = q / 9;
    const int64_t fb = fbk[(ix ? 1 : 0) | (iy ? 2 : 0) | (iz ? 4 : 0)];
    const int fc = node_cell(px[ix], py[iy], pz[iz]);
    const float w = 1.f / float(wx[ix] * wy[iy] * wz[iz]);
    const float* sd = a.lam_fine + fb * kBlockVals + fc;
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = fmaf(w, sd[r * kCells], acc[r]);
  }
  const float lu[3] = {acc[1], acc[2], acc[3]};
  const float lsn[6] = {acc[4], acc[5], acc[6], acc[7], acc[8], acc[9]};
  float m[kRows], dl[kRows];
  load_f32(a.coarse.mom_other, cb, cc, m);
  split_adjoint(m, a.avg ? 0.5f : 1.f, acc[0], lu, lsn, dl);
  add10(a.lam_old + cb * kBlockVals + cc, dl);
  if (a.avg) {
    load_f32(a.coarse.mom, cb, cc, m);
    split_adjoint(m, 0.5f, acc[0], lu, lsn, dl);
    add_lambda(a.lam_new, cb, cc, dl);
  }
}

// Set-up of the gather, once per adjoint: bit of every I^d node of the fine
// level, and bit of every coarse node that an I^d stencil holds.
__global__ void k_mark_down(DownAdjArgs a, uint32_t* __restrict__ fine_bits, uint32_t* __restrict__ coarse_bits) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n_nodes) return;
  const int32_t v = a.nodes[k];
  const int64_t b = v >> 9;
  const int cell = v & 511;
  atomicOr(fine_bits + b * (kCells / 32) + (cell >> 5), 1u << (cell & 31));
  const int32_t* c = a.fine.coords + 3 * b;
  const int p[3] = {c[0] * 8 + (cell & 7), c[1] * 8 + ((cell >> 3) & 7), c[2] * 8 + (cell >> 6)};
  const int n[3] = {a.coarse.d.nx * 8, a.coarse.d.ny * 8, a.coarse.d.nz * 8};
  int lo[3], hi[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) stencil_axis(p[ax], n[ax], a.periodic[ax], lo[ax], hi[ax]);
  for (int q = 0; q < 8; ++q) {
    const int x = (q & 1) ? hi[0] : lo[0], y = (q & 2) ? hi[1] : lo[1], z = (q & 4) ? hi[2] : lo[2];
    const int64_t cb = find_block(a.coarse, x, y, z);
    if (cb < 0) continue;
    const int cc = node_cell(x, y, z);
    atomicOr(coarse_bits + cb * (kCells / 32) + (cc >> 5), 1u << (cc & 31));
  }
}

// Set bits of a level's node bitmap listed as (block << 9) | cell, in block
// order: per-block counts, one exclusive scan, then the scatter.
__global__ void __launch_bounds__(kCells) k_bits_count(const uint32_t* __restrict__ bits, int64_t* __restrict__ counts) {
  __shared__ int s_cnt[kCells / 32];
  const int64_t b = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_cnt[w] = __popc(bits[b * (kCells / 32) + w]);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int i = 0; i < kCells / 32; ++i) s += s_cnt[i];
    counts[b] = s;
  }
}

__global__ void __launch_bounds__(1024) k_counts_scan(int64_t* __restrict__ counts, int64_t nb,
                                                      int64_t* __restrict__ total) {
  __shared__ int64_t s_part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = min(nb, int64_t(t) * per), b1 = min(nb, b0 + per);
  int64_t sum = 0;
  for (int64_t b = b0; b < b1; ++b) sum += counts[b];
  s_part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int i = 0; i < int(blockDim.x); ++i) {
      const int64_t c = s_part[i];
      s_part[i] = run;
      run += c;
    }
    *total = run;
  }
  __syncthreads();
  int64_t run = s_part[t];
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t c = counts[b];
    counts[b] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kCells) k_bits_scatter(const uint32_t* __restrict__ bits,
                                                         const int64_t* __restrict__ offs, int32_t* __restrict__ out) {
  __shared__ int s_off[kCells / 32];
  const int64_t b = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t word = bits[b * (kCells / 32) + w];
  if (lane == 0) s_off[w] = __popc(word);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int i = 0; i < kCells / 32; ++i) {
      const int c = s_off[i];
      s_off[i] = s;
      s += c;
    }
  }
  __syncthreads();
  if (!((word >> lane) & 1u)) return;
  out[offs[b] + s_off[w] + __popc(word & ((1u << lane) - 1u))] = int32_t((b << 9) | threadIdx.x);
}

struct UpAdjArgs {
  LevelView fine, coarse;  // fine.mom = A_l as the upward transfer read it
  const int32_t* nodes;    // I^u_{l+1}: (block << 9) | cell of the coarse level
  int64_t n_nodes;
  float k;                 // S^neq factor of the transfer
  LamTarget lam_fine;      // lambda_A_l
  float* lam_coarse;       // lambda_A_{l+1} at pass-through nodes: read at I^u, then zeroed
};

// Transposed upward transfer: the coarse node stores (rho_f - 1, u_f,
// k S_f + (1 - k) u_f u_f) of its coincident fine node, which no other coarse
// node reads, so the fine adjoint is updated without atomics.
__global__ void k_up_adj(UpAdjArgs a) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n_nodes) return;
  const int32_t v = a.nodes[k];
  const int64_t b = v >> 9;
  const int cell = v & 511;
  const int32_t* c = a.coarse.coords + 3 * b;
  const int x = 2 * (c[0] * 8 + (cell & 7)), y = 2 * (c[1] * 8 + ((cell >> 3) & 7)), z = 2 * (c[2] * 8 + (cell >> 6));
  const int64_t fb = find_block(a.fine, x, y, z);
  if (fb < 0) return;
  float* lc = a.lam_coarse + b * kBlockVals + cell;
  float L[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    L[r] = lc[r * kCells];
    lc[r * kCells] = 0.f;
  }
  const int fc = node_cell(x, y, z);
  float m[kRows];
  load_f32(a.fine.mom, fb, fc, m);
  const float ux = m[1], uy = m[2], uz = m[3], e = 1.f - a.k;
  float dl[kRows];
  dl[0] = L[0];
  dl[1] = L[1] + e * (2.f * ux * L[4] + uy * L[7] + uz * L[8]);
  dl[2] = L[2] + e * (2.f * uy * L[5] + ux * L[7] + uz * L[9]);
  dl[3] = L[3] + e * (2.f * uz * L[6] + ux * L[8] + uy * L[9]);
#pragma unroll
  for (int r = 4; r < kRows; ++r) dl[r] = a.k * L[r];
  add_lambda(a.lam_fine, fb, fc, dl);
}

// Undo log of the transfers (written by the transfer kernels during the
// recomputation, [n][10] in the order of nodes): puts the logged values back;
// lam, if set, is zeroed at the same nodes (natural order).
__global__ void k_scatter_nodes(float* __restrict__ buf, const int32_t* __restrict__ nodes, int64_t n,
                                const float* __restrict__ log, float* __restrict__ lam) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int32_t v = nodes[k];
  float* p = buf + int64_t(v >> 9) * kBlockVals + node_offset<float>(v & 511);
#pragma unroll
  for (int r = 0; r < kRows; ++r) p[r * kCells] = log[k * kRows + r];
  if (lam != nullptr) {
    float* q = lam + int64_t(v >> 9) * kBlockVals + (v & 511);
#pragma unroll
    for (int r = 0; r < kRows; ++r) q[r * kCells] = 0.f;
  }
}

inline unsigned grid_for(int64_t n) { return unsigned((n + 255) / 256); }

// ---------------------------------------------------------------- host driver

using Op = AdjOp;  // pointers as the forward recomputation used them

// The operations of one coarse step, in the order of AdvanceLBM (Algorithm 1).
void coarse_step_ops(int L, int l, int s, std::vector<Op>& ops) {
  if (l < L - 1) ops.push_back(Op{kDown, l, s});
  ops.push_back(Op{kSC, l, 0});
  if (l < L - 1 && s == 2) ops.push_back(Op{kUp, l, 0});
  if (l > 0) {
    coarse_step_ops(L, l - 1, 1, ops);
    coarse_step_ops(L, l - 1, 2, ops);
  }
}

GridDims level_dims(const hlbm_lattice* h, int l) {
  int d[3];
  h->block_dims(l, d);
  return GridDims{d[0], d[1], d[2]};
}

LevelView level_view(const hlbm_lattice* h, int l, const void* mom, const void* other) {
  const LevelData& L = h->lv[l];
  LevelView v{};
  v.d = level_dims(h, l);
  v.slot = L.d_slot;
  v.hash = BlockHash{L.d_hkeys, L.d_hvals, L.hcap ? L.hcap - 1u : 0u};
  v.coords = L.d_coords;
  v.mom = mom;
  v.mom_other = other;
  v.nb = L.nb;
  v.sc = nullptr;
  return v;
}

StepArgs level_args(const hlbm_lattice* h, int l) {
  const LevelData& L = h->lv[l];
  StepArgs a{};
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
  return a;
}

// The operations of one checkpoint segment (k_coarse coarse steps) with
// their buffers, the per-level working copies of the segment's start state
// and the FP64 sums of the recomputed downward transfers.  get(bytes, &p)
// allocates and keeps the allocation.
template <class Get>
int alloc_segment(hlbm_lattice* h, int k_coarse, Get&& get, std::vector<Op>& seg_ops, std::vector<void*>& work,
                  std::vector<double*>& acc) {
  const int L = h->cfg.num_levels;
  std::vector<Op> step_ops;
  coarse_step_ops(L, L - 1, 1, step_ops);
  seg_ops.clear();
  for (int c = 0; c < k_coarse; ++c) seg_ops.insert(seg_ops.end(), step_ops.begin(), step_ops.end());
  work.assign(size_t(L), nullptr);
  acc.assign(size_t(L), nullptr);
  void* p;
  for (int l = 0; l < L; ++l)
    if (int rc = get(size_t(h->lv[l].nb) * kBlockVals * sizeof(float), &work[size_t(l)])) return rc;
  for (int l = 0; l + 1 < L; ++l) {
    if (int rc = get((size_t(h->lv[l].n_down) * 10 + 1) * sizeof(double), &p)) return rc;
    acc[size_t(l)] = static_cast<double*>(p);
  }
  for (Op& op : seg_ops) {
    if (op.kind == kSC) {
      if (int rc = get(size_t(h->lv[op.l].nb) * kBlockVals * sizeof(float), &op.out)) return rc;
      if (int rc = get(size_t(h->lv[op.l].nb) * kBlockVals * sizeof(float), &p)) return rc;
      op.pre = static_cast<float*>(p);
    } else {
      const int64_t n = op.kind == kDown ? h->lv[op.l].n_down : h->lv[op.l + 1].n_up;
      if (int rc = get(size_t(n) * kRows * sizeof(float), &p)) return rc;
      op.undo = static_cast<float*>(p);
    }
  }
  return HLBM_OK;
}

// Runs the first n_ops operations of a segment from the per-level start
// states start[l] (copied into work first), recording every SC's p, logging
// what the transfers overwrite and keeping each operation's buffers in its
// record; cur[l] ends as the level's final state.
cudaError_t recompute_segment(hlbm_lattice* h, std::vector<Op>& seg_ops, size_t n_ops, const std::vector<void*>& start,
                              const std::vector<void*>& work, const std::vector<double*>& acc, std::vector<void*>& cur) {
  const int L = h->cfg.num_levels;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  std::vector<void*> prev(size_t(L), nullptr);
  cur.assign(size_t(L), nullptr);
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    const size_t vals = size_t(h->lv[l].nb) * kBlockVals;
    if (vals) e = cudaMemcpyAsync(work[size_t(l)], start[size_t(l)], vals * sizeof(float), cudaMemcpyDeviceToDevice, st);
    cur[size_t(l)] = work[size_t(l)];
  }
  for (size_t i = 0; i < n_ops && e == cudaSuccess; ++i) {
    Op& op = seg_ops[i];
    const int l = op.l;
    if (op.kind == kSC) {
      if (h->lv[l].nb == 0) {
        prev[l] = cur[l];
        continue;
      }
      StepArgs a = level_args(h, l);
      a.in = cur[l];
      a.out = op.out;
      a.pre_out = op.pre;
      e = launch_stream_collide_record(a, st);
      op.in = cur[l];
      prev[l] = cur[l];
      cur[l] = op.out;
    } else if (op.kind == kDown) {
      const LevelData& F = h->lv[l];
      op.in = cur[l];
      op.c_old = prev[l + 1];
      op.c_new = cur[l + 1];
      if (F.n_down == 0) continue;
      TransferArgs t{};
      t.undo = op.undo;  // in transfer order
      t.fine = level_view(h, l, cur[l], nullptr);
      t.coarse = level_view(h, l + 1, cur[l + 1], prev[l + 1]);
      t.out = cur[l];
      t.nodes = F.d_down_t;
      t.stencil = F.d_down_stc;
      t.n_nodes = F.n_down;
      t.avg = op.s == 2 ? 1 : 0;
      t.use_other = op.s == 1 ? 1 : 0;
      t.acc_old = acc[size_t(l)];
      t.k = h->kdown[l];
      for (int ax = 0; ax < 3; ++ax) t.periodic[ax] = h->cfg.periodic[ax];
      t.status = h->d_status;
      e = transfer_down(HLBM_STORE_F32, t, st);
    } else {
      const LevelData& C = h->lv[l + 1];
      op.in = cur[l + 1];
      op.c_new = cur[l];
      if (C.n_up == 0) continue;
      TransferArgs t{};
      t.undo = op.undo;
      t.fine = level_view(h, l, cur[l], nullptr);
      t.coarse = level_view(h, l + 1, cur[l + 1], nullptr);
      t.out = cur[l + 1];
      t.nodes = C.d_up;
      t.n_nodes = C.n_up;
      t.k = h->kup[l];
      for (int ax = 0; ax < 3; ++ax) t.periodic[ax] = h->cfg.periodic[ax];
      t.status = h->d_status;
      e = transfer_up(HLBM_STORE_F32, t, st);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  return e;
}

}  // namespace

int ml_forward_record(hlbm_lattice* h, int32_t n_steps, int32_t ckpt_every) {
  const int L = h->cfg.num_levels;
  const int32_t per = 1 << (L - 1);
  if (h->cfg.storage != HLBM_STORE_F32)
    return fail(h, HLBM_E_UNSUPPORTED, "the adjoint of a multi-level or sparse lattice needs FP32 storage");
  if (n_steps % per != 0 || ckpt_every % per != 0)
    return fail(h, HLBM_E_INVALID_ARG, "n_steps and ckpt_every must be multiples of %d fine steps", per);
  const int32_t n_coarse = n_steps / per, k_coarse = ckpt_every / per;
  const int n_ck = (n_coarse + k_coarse - 1) / k_coarse;
  int rc;
  for (int c = 0; c < n_ck; ++c)
    for (int l = 0; l < L; ++l) {
      void* p = nullptr;
      if ((rc = LatticeOps::alloc(h, &p, size_t(h->lv[l].nb) * kBlockVals * sizeof(float)))) return rc;
      h->ckpt.push_back(p);
    }
  // the tape of the last segment, allocated before anything runs
  AdjTape* tape = new AdjTape();
  h->tape = tape;
  auto get = [&](size_t bytes, void** out) -> int {
    *out = nullptr;
    const int r = LatticeOps::alloc(h, out, bytes);
    if (r == HLBM_OK && *out != nullptr) tape->bufs.push_back(*out);
    return r;
  };
  if ((rc = alloc_segment(h, k_coarse, get, tape->ops, tape->work, tape->acc))) return rc;
  const int32_t t_last = (n_ck - 1) * k_coarse;
  for (int32_t t = 0; t <= t_last; ++t) {
    if (t % k_coarse == 0)
      for (int l = 0; l < L; ++l) {
        const LevelData& Lv = h->lv[l];
        if (Lv.nb == 0) continue;
        const cudaError_t e = cudaMemcpyAsync(h->ckpt[size_t(t / k_coarse) * L + l], Lv.d_mom[Lv.cur],
                                              size_t(Lv.nb) * kBlockVals * sizeof(float), cudaMemcpyDeviceToDevice,
                                              h->stream);
        if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "checkpoint copy: %s", cudaGetErrorString(e));
      }
    if (t < t_last && (rc = ml_advance_coarse(h, 1))) return rc;
  }
  // the last segment: the adjoint's recomputation, from the last checkpoint,
  // kept as the tape; its final states become the lattice's state
  tape->n = n_coarse - t_last;
  std::vector<Op> step_ops;
  coarse_step_ops(L, L - 1, 1, step_ops);
  std::vector<void*> start(static_cast<size_t>(L)), cur;
  for (int l = 0; l < L; ++l) start[size_t(l)] = h->ckpt[size_t(n_ck - 1) * L + l];
  cudaError_t e = recompute_segment(h, tape->ops, size_t(tape->n) * step_ops.size(), start, tape->work, tape->acc, cur);
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    LevelData& Lv = h->lv[l];
    if (Lv.nb)
      e = cudaMemcpyAsync(Lv.d_mom[Lv.cur], cur[size_t(l)], size_t(Lv.nb) * kBlockVals * sizeof(float),
                          cudaMemcpyDeviceToDevice, h->stream);
  }
  if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "recording the last segment: %s", cudaGetErrorString(e));
  h->l0_steps += int64_t(tape->n) * per;
  h->rec_steps = n_steps;
  h->rec_every = ckpt_every;
  return ml_check_status(h);
}

int ml_adjoint(hlbm_lattice* h, const float* dL_dM, float* dL_dF) {
  const int L = h->cfg.num_levels;
  const int32_t per = 1 << (L - 1);
  const int32_t n_coarse = h->rec_steps / per, k_coarse = h->rec_every / per;
  const int n_seg = (n_coarse + k_coarse - 1) / k_coarse;
  std::vector<size_t> vals(L);
  size_t vmax = 0;
  for (int l = 0; l < L; ++l) {
    vals[l] = size_t(h->lv[l].nb) * kBlockVals;
    if (vals[l] > vmax) vmax = vals[l];
  }
  std::vector<void*> tmp;
  auto release_all = [&]() {
    for (void*& p : tmp) LatticeOps::release(h, p);
  };
  int rc = HLBM_OK;
  auto get = [&](size_t bytes, void** out) -> int {
    *out = nullptr;
    if (rc != HLBM_OK) return rc;
    rc = LatticeOps::alloc(h, out, bytes);
    if (rc == HLBM_OK && *out != nullptr) tmp.push_back(*out);
    return rc;
  };
  // one coarse step's operations; the segment repeats them
  std::vector<Op> step_ops;
  coarse_step_ops(L, L - 1, 1, step_ops);
  // adjoints (each sized for the largest level, so that buffers can swap)
  std::vector<float*> lamA(L), lamP(L);
  float *spare = nullptr, *lamp = nullptr;
  // dL/dF: an FP32 sum per checkpoint segment (dFs), added to the FP64 sum
  // over segments (dF) when the segment is done
  double* dF = nullptr;
  float* dFs = nullptr;
  for (int l = 0; l < L; ++l) {
    void* p;
    get(vmax * sizeof(float), &p);
    lamA[l] = static_cast<float*>(p);
    get(vmax * sizeof(float), &p);
    lamP[l] = static_cast<float*>(p);
  }
  {
    void* p;
    get(vmax * sizeof(float), &p);
    spare = static_cast<float*>(p);
    get(vmax * sizeof(float), &p);
    lamp = static_cast<float*>(p);
    get(size_t(h->lv[0].nb) * 3 * kCells * sizeof(double), &p);
    dF = static_cast<double*>(p);
    get(size_t(h->lv[0].nb) * 3 * kCells * sizeof(float), &p);
    dFs = static_cast<float*>(p);
  }
  // segment buffers (working copies of the checkpoint, one output and one
  // pre-collision buffer per SC operation, undo logs per transfer, the FP64
  // sums of the recomputed downward transfers): the recording's tape when
  // there is one, else allocated here
  std::vector<Op> seg_ops;
  std::vector<void*> work;
  std::vector<double*> acc;
  AdjTape* tape = h->tape;
  if (tape != nullptr) {
    seg_ops = tape->ops;
    work = tape->work;
    acc = tape->acc;
  } else {
    alloc_segment(h, k_coarse, get, seg_ops, work, acc);
  }
  // lambda at the pass-through nodes of a fused level, and the pass-through bits
  std::vector<float*> raw(L, nullptr);
  std::vector<uint32_t*> ptb(L, nullptr);
  for (int l = 0; l < L; ++l) {
    void* p;
    get(vals[l] * sizeof(float), &p);
    raw[l] = static_cast<float*>(p);
    get(size_t(h->lv[l].nb) * (kCells / 32) * sizeof(uint32_t) + sizeof(uint32_t), &p);
    ptb[l] = static_cast<uint32_t*>(p);
  }
  // the level's previous SC in the segment, for every SC (-1: the first)
  std::vector<int> prev_sc(seg_ops.size(), -1);
  {
    std::vector<int> last(L, -1);
    for (size_t i = 0; i < seg_ops.size(); ++i)
      if (seg_ops[i].kind == kSC) {
        prev_sc[i] = last[seg_ops[i].l];
        last[seg_ops[i].l] = int(i);
      }
  }
  if (rc != HLBM_OK) {
    release_all();
    return rc;
  }
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  size_t off = 0;
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    if (vals[l]) e = cudaMemcpyAsync(lamA[l], dL_dM + off, vals[l] * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && vals[l]) e = cudaMemsetAsync(lamP[l], 0, vals[l] * sizeof(float), st);
    off += vals[l];
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(dF, 0, size_t(h->lv[0].nb) * 3 * kCells * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dFs, 0, size_t(h->lv[0].nb) * 3 * kCells * sizeof(float), st);
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    const LevelData& Lv = h->lv[l];
    if (Lv.nb == 0) continue;
    k_passthrough_bits<<<unsigned(Lv.nb), kCells, 0, st>>>(Lv.d_nbr, Lv.d_bflags, Lv.d_solid, ptb[l]);
    e = cudaGetLastError();
  }
  // The gather of the transposed downward transfers: per level pair, the I^d
  // bits of the fine level and the list of coarse nodes the I^d stencils hold
  std::vector<uint32_t*> fbits(L, nullptr);
  std::vector<int32_t*> tgt(L, nullptr);
  std::vector<int64_t> n_tgt(L, 0);
  {
    std::vector<uint32_t*> cbits(L, nullptr);
    std::vector<int64_t*> cnt(L, nullptr);
    int64_t* d_tot = nullptr;
    void* p;
    if (get(size_t(L) * sizeof(int64_t), &p) == HLBM_OK) d_tot = static_cast<int64_t*>(p);
    for (int l = 0; l + 1 < L && rc == HLBM_OK; ++l) {
      const LevelData &F = h->lv[l], &C = h->lv[l + 1];
      if (F.n_down == 0 || C.nb == 0) continue;
      if (get(size_t(F.nb) * (kCells / 32) * sizeof(uint32_t), &p)) break;
      fbits[l] = static_cast<uint32_t*>(p);
      if (get(size_t(C.nb) * (kCells / 32) * sizeof(uint32_t), &p)) break;
      cbits[l] = static_cast<uint32_t*>(p);
      if (get(size_t(C.nb) * sizeof(int64_t), &p)) break;
      cnt[l] = static_cast<int64_t*>(p);
    }
    for (int l = 0; l + 1 < L && rc == HLBM_OK && e == cudaSuccess; ++l) {
      if (cnt[l] == nullptr) continue;
      const LevelData &F = h->lv[l], &C = h->lv[l + 1];
      e = cudaMemsetAsync(fbits[l], 0, size_t(F.nb) * (kCells / 32) * sizeof(uint32_t), st);
      if (e == cudaSuccess) e = cudaMemsetAsync(cbits[l], 0, size_t(C.nb) * (kCells / 32) * sizeof(uint32_t), st);
      if (e != cudaSuccess) break;
      DownAdjArgs d{};
      d.fine = level_view(h, l, nullptr, nullptr);
      d.coarse = level_view(h, l + 1, nullptr, nullptr);
      d.nodes = F.d_down;
      d.n_nodes = F.n_down;
      for (int ax = 0; ax < 3; ++ax) d.periodic[ax] = h->cfg.periodic[ax];
      k_mark_down<<<grid_for(F.n_down), 256, 0, st>>>(d, fbits[l], cbits[l]);
      k_bits_count<<<unsigned(C.nb), kCells, 0, st>>>(cbits[l], cnt[l]);
      k_counts_scan<<<1, 1024, 0, st>>>(cnt[l], C.nb, d_tot + l);
      e = cudaGetLastError();
    }
    std::vector<int64_t> tot(size_t(L), 0);
    if (rc == HLBM_OK && e == cudaSuccess) e = cudaMemcpyAsync(tot.data(), d_tot, L * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (rc == HLBM_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int l = 0; l + 1 < L && rc == HLBM_OK && e == cudaSuccess; ++l) {
      if (cnt[l] == nullptr || tot[size_t(l)] == 0) continue;
      if (get(size_t(tot[size_t(l)]) * sizeof(int32_t), &p)) break;
      tgt[l] = static_cast<int32_t*>(p);
      n_tgt[l] = tot[size_t(l)];
      k_bits_scatter<<<unsigned(h->lv[l + 1].nb), kCells, 0, st>>>(cbits[l], cnt[l], tgt[l]);
      e = cudaGetLastError();
    }
    if (rc != HLBM_OK) {
      release_all();
      return rc;
    }
  }
  // every allocation went through: the adjoint takes the tape over (its
  // reverse walk changes the tape's buffers; they are released with the rest)
  const bool taped = tape != nullptr;
  if (taped) {
    tmp.insert(tmp.end(), tape->bufs.begin(), tape->bufs.end());
    delete tape;
    h->tape = nullptr;
  }
  // Per level: plain (lamA holds lambda) or fused (lamA holds mu, raw holds
  // lambda at the pass-through nodes; fpre is the recorded p of the level's
  // next SC to reverse, whose transposed collision mu already includes).
  // Within a segment every SC but the level's first is reversed fused with
  // the transposed collision of the SC before it.
  std::vector<char> fused(L, 0);
  std::vector<const float*> fpre(L, nullptr);
  auto target = [&](int l) {
    LamTarget g{};
    if (!fused[l]) {
      g.raw = lamA[l];
      return g;
    }
    const StepArgs a = level_args(h, l);
    g.pt = ptb[l];
    g.raw = raw[l];
    g.mu = lamA[l];
    g.pre = fpre[l];
    g.F = a.F;
    g.eps = a.eps;
    for (int ax = 0; ax < 3; ++ax) g.fu[ax] = float(a.fu[ax]);
    g.om = float(a.om);
    g.tau = float(a.tau);
    g.dF = l == 0 ? dFs : nullptr;
    return g;
  };

  for (int sgi = n_seg - 1; sgi >= 0 && e == cudaSuccess; --sgi) {
    const int nc = (n_coarse - sgi * k_coarse) < k_coarse ? (n_coarse - sgi * k_coarse) : k_coarse;
    const size_t n_ops = size_t(nc) * step_ops.size();
    // 1. recompute the segment from its checkpoint, logging what every
    // operation read (the last segment: the recording's tape holds it)
    if (!(taped && sgi == n_seg - 1)) {
      std::vector<void*> start(static_cast<size_t>(L)), cur;
      for (int l = 0; l < L; ++l) start[size_t(l)] = h->ckpt[size_t(sgi) * L + l];
      e = recompute_segment(h, seg_ops, n_ops, start, work, acc, cur);
    }
    // 2. walk the operations backwards
    for (size_t i = n_ops; i-- > 0 && e == cudaSuccess;) {
      const Op& op = seg_ops[i];
      const int l = op.l;
      if (op.kind == kSC) {
        if (h->lv[l].nb == 0) continue;
        StepArgs a = level_args(h, l);
        a.in = op.in;
        const float* lp_in = lamA[l];  // lambda_p of this SC
        const float* pass = raw[l];    // lambda at its pass-through nodes
        if (!fused[l]) {
          e = adjoint_collide(a, op.pre, lamA[l], lamp, nullptr, st, l == 0 ? dFs : nullptr);
          lp_in = lamp;
          pass = lamA[l];
        }
        // lambda_P is added and left zero by the same pass; lambda_P of level 0
        // stays zero (no finer level reads its previous state)
        float* add = l > 0 ? lamP[l] : nullptr;
        if (e == cudaSuccess && prev_sc[i] >= 0) {
          const float* pp = seg_ops[size_t(prev_sc[i])].pre;
          e = adjoint_push_collide(a, lp_in, pp, spare, nullptr, st, pass, raw[l], add, true, l == 0 ? dFs : nullptr);
          fused[l] = 1;
          fpre[l] = pp;
        } else if (e == cudaSuccess) {
          e = adjoint_push(a, pass, lp_in, spare, st, add, true);
          fused[l] = 0;
        }
        std::swap(lamA[l], spare);
      } else if (op.kind == kDown) {
        const LevelData& F = h->lv[l];
        if (F.n_down == 0) continue;
        DownAdjArgs d{};
        d.fine = level_view(h, l, op.in, nullptr);
        d.coarse = level_view(h, l + 1, op.c_new, op.c_old);
        d.nodes = F.d_down_t;  // the seeds are per node: transfer order (uniform stencil shape per warp)
        d.stencil = F.d_down_stc;
        d.n_nodes = F.n_down;
        d.avg = op.s == 2 ? 1 : 0;
        d.k = float(h->kdown[l]);
        for (int ax = 0; ax < 3; ++ax) d.periodic[ax] = h->cfg.periodic[ax];
        d.lam_fine = fused[l] ? raw[l] : lamA[l];
        d.lam_new = target(l + 1);
        d.lam_old = lamP[l + 1];
        k_down_adj_seed<<<grid_for(F.n_down), 256, 0, st>>>(d);
        if (n_tgt[l] > 0) k_down_adj_gather<<<grid_for(n_tgt[l]), 256, 0, st>>>(d, tgt[l], n_tgt[l], fbits[l]);
        k_scatter_nodes<<<grid_for(F.n_down), 256, 0, st>>>(static_cast<float*>(op.in), F.d_down_t, F.n_down,
                                                            op.undo, d.lam_fine);
      } else {
        const LevelData& C = h->lv[l + 1];
        if (C.n_up == 0) continue;
        UpAdjArgs u{};
        u.fine = level_view(h, l, op.c_new, nullptr);
        u.coarse = level_view(h, l + 1, op.in, nullptr);
        u.nodes = C.d_up;
        u.n_nodes = C.n_up;
        u.k = float(h->kup[l]);
        u.lam_fine = target(l);
        u.lam_coarse = fused[l + 1] ? raw[l + 1] : lamA[l + 1];
        k_up_adj<<<grid_for(C.n_up), 256, 0, st>>>(u);
        k_scatter_nodes<<<grid_for(C.n_up), 256, 0, st>>>(static_cast<float*>(op.in), C.d_up, C.n_up, op.undo,
                                                          nullptr);
      }
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = adjoint_dF_flush(dF, dFs, h->lv[0].nb * 3 * kCells, st);
  }
  if (e == cudaSuccess)
    e = adjoint_dF_to_float(dF, dL_dF, h->lv[0].nb * 3 * kCells, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release_all();
  if (e != cudaSuccess) return fail(h, HLBM_E_CUDA, "adjoint: %s", cudaGetErrorString(e));
  return ml_check_status(h);
}

}  // namespace hlbm
