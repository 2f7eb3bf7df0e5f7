/*
 * homelbm.h -- C ABI of the GB300 moment-encoded multi-level lattice Boltzmann
 * hot path (libhomelbm.so).
 *
 * The library advances the moment set M = {rho, u, S} of the paper's HOME-LBM
 * scheme (Sec. 3.1, Eq. rho_u_stress and Eq. three_order_f) on a block-sparse,
 * multi-level D3Q27 lattice (Sec. 5.1, Sec. 6.1), with the sub-cycled advance of
 * Algorithm 1 and the fine<->coarse transfers of Eq. downward_rescale and
 * Eq. upload_S, and rebuilds the block hierarchy from a particle cloud through
 * the level-selection function Phi (Sec. 5.4, Sec. 6.3).
 *
 * Conventions
 *  - Every call returns an hlbm_status (int32).  Nothing aborts and no C++
 *    exception crosses the ABI.  hlbm_last_error() gives a message owned by the
 *    handle (valid until the next call on that handle).
 *  - A handle is not thread-safe; calls on one handle must be serialised.
 *  - All device work is enqueued on the stream given in hlbm_config (borrowed,
 *    never destroyed; NULL = the legacy default stream).  Calls that return
 *    data to host memory synchronise that stream.
 *  - Blocks are cubes of 8^3 nodes.  A block-major field of one level has the
 *    layout [n_blocks][rows][512] with the node index x + 8 y + 64 z inside the
 *    block, blocks in ascending linear slot id bz*(nby*nbx) + by*nbx + bx.
 *  - Moment rows: 0 rho, 1 u_x, 2 u_y, 3 u_z, 4 S_xx, 5 S_yy, 6 S_zz, 7 S_xy,
 *    8 S_xz, 9 S_yz.  The stored set is the POST-collision one, so the stored
 *    velocity is u' = u + F/(2 rho) (Eq. rho_u_stress read with Guo forcing).
 *  - Level 0 is the finest.  A node of level l sits at fine position
 *    2^l * index (vertex-aligned levels).
 */
#ifndef HOMELBM_H
#define HOMELBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HLBM_OK = 0,
  HLBM_E_INVALID_ARG = 1, /* bad pointer, size, level or configuration */
  HLBM_E_BAD_STATE = 2,   /* call out of order, e.g. step before blocks are set */
  HLBM_E_OOM = 3,         /* device or host allocation failed */
  HLBM_E_CUDA = 4,        /* a CUDA runtime call failed; message has the CUDA error */
  HLBM_E_NONFINITE = 5,   /* an input field or a reduction is not finite */
  HLBM_E_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  HLBM_E_UNSUPPORTED = 7  /* valid request the library does not implement */
} hlbm_status;

typedef enum {
  HLBM_STORE_F64 = 0,   /* 80 B per node */
  HLBM_STORE_F32 = 1,   /* 40 B per node */
  HLBM_STORE_F16S = 2,  /* 20 B per node: fp16 x per-row power-of-two scale */
  HLBM_STORE_BF16S = 3  /* 20 B per node: bf16 x per-row power-of-two scale */
} hlbm_storage;

typedef enum {
  /* S^neq of the stored post-collision moments scales with (tau-1) times the
     lattice velocity gradient: k_up = 2 (tau_c-1)/(tau_f-1), k_down = 1/k_up.
     The factor changes sign where the levels' tau lie on both sides of 1 and
     grows without bound as a level's tau approaches 1: hlbm_create refuses
     (HLBM_E_INVALID_ARG) a tau_finest whose factors leave [1/100, 100] in
     magnitude for FP32, FP16 and BF16 storage ([1e-6, 1e6] for FP64), since
     the transfers multiply the rounding of the stored S by |k|. */
  HLBM_RESCALE_POST = 0,
  /* Chapman-Enskog scaling of the pre-collision S^neq: k_up = 2 tau_c/tau_f. */
  HLBM_RESCALE_PRE = 1,
  /* factors as printed in Eq. upload_S (tau_c/(2 tau_f)) and
     Eq. downward_rescale (2 tau_c/tau_f). */
  HLBM_RESCALE_PAPER = 2
} hlbm_rescale;

typedef struct {
  int32_t nx, ny, nz;      /* fine-equivalent extent; multiples of 8*2^(L-1) */
  int32_t block_edge;      /* must be 8 */
  int32_t num_levels;      /* L >= 1 */
  double tau_finest;       /* tau_0 > 1/2; tau_{l+1} = tau_l/2 + 1/4 (Sec. 5.2) */
  int32_t periodic[3];     /* per axis x, y, z; non-periodic faces are half-way bounce-back walls */
  int32_t storage;         /* hlbm_storage */
  int32_t rescale_mode;    /* hlbm_rescale */
  int32_t xyz_literal;     /* 0: third-order xyz weight 1/c_s^6 (Hermite series);
                              1: 1/(2 c_s^6) as printed after Eq. three_order_f */
  void *stream;            /* cudaStream_t, borrowed: every kernel, copy and device
                              allocation of the handle is ordered on it (device
                              buffers come from the stream-ordered pool), so it
                              must stay valid until hlbm_destroy returns */
  int32_t device;          /* CUDA device ordinal */
} hlbm_config;

typedef struct hlbm_lattice hlbm_lattice;

/* Face conditions of hlbm_set_open_faces. */
typedef enum {
  HLBM_FACE_CLOSED = 0,   /* periodic or half-way bounce-back wall, as the axis is configured */
  HLBM_FACE_OUTFLOW = 1,  /* convective outflow dM/dt + u_n dM/dn = 0 */
  HLBM_FACE_INLET = 2     /* logarithmic inlet profile */
} hlbm_face;

/* Library version string (static). */
const char *hlbm_version(void);

/* Create a lattice.  No blocks are stored until hlbm_set_blocks,
   hlbm_set_dense or hlbm_rebuild_from_particles.  *out is NULL on failure. */
int32_t hlbm_create(const hlbm_config *cfg, hlbm_lattice **out);

/* Free every device and host resource of the handle.  NULL is accepted. */
int32_t hlbm_destroy(hlbm_lattice *h);

/* Message of the last failed call on h (or of the last failed hlbm_create when
   h is NULL).  Owned by the library. */
const char *hlbm_last_error(const hlbm_lattice *h);

/* Store every block of a single-level lattice (L must be 1).  Moments are set
   to rest (rho = 1, u = 0, S = 0). */
int32_t hlbm_set_dense(hlbm_lattice *h);

/* Declare the level-0 blocks that must be resolved at the finest level (the
   blocks where the level-selection function Phi of Sec. 5.4 is 0) and build
   the whole hierarchy from them on the device (same pipeline as
   hlbm_rebuild_from_particles).  coords_xyz: host int32 [n][3] block
   coordinates (bx, by, bz) of level 0.  On the first call every stored node is
   at rest; later calls carry the moments over like a rebuild. */
int32_t hlbm_set_fine_blocks(hlbm_lattice *h, const int32_t *coords_xyz, int64_t n);

/* Set the block hierarchy explicitly, one level per call (Sec. 5.1 and 6.1:
   each level stores its leaf and border blocks; Sec. 5.3: neighbouring
   levels overlap and levels two apart are separated).  coords_xyz: host
   int32 [n][3] block coordinates (bx, by, bz) of the blocks stored at
   `level` (block edge 8 << level fine nodes), copied; any order.  The call
   that stages the last level not yet staged since the previous explicit
   hierarchy validates all levels and installs them like a rebuild: block
   lists in ascending slot order, flags against the previous hierarchy,
   neighbour tables and interface nodes, moments carried over (every node at
   rest on the first hierarchy).  With H_l the level-l blocks whose children
   are stored or internal and I_l the blocks of H_l whose 26 in-domain
   neighbours are all in H_l, the hierarchy must satisfy, else
   HLBM_E_INVALID_ARG (message names the first failing block), the staged
   lists are dropped and the lattice keeps its previous state:
   - every coordinate inside the level's block grid, no block listed twice;
   - no stored block is internal (in I_l);
   - every stored block below the top has a parent that is stored or internal;
   - every child of a block in H_{l+1} is stored or internal, and the top
     level stores every block that is not internal;
   - overlap and separation: H_l is a union of 3x3x3-block cubes (H_l equals
     the one-block dilation of I_l), so every refined region keeps one coarse
     block of overlap;
   - 2:1 grading: H_{l+1} contains the one-block dilation of parent(H_l).
   Every hierarchy hlbm_rebuild_from_particles builds passes.  Synchronous. */
int32_t hlbm_set_blocks(hlbm_lattice *h, int32_t level, const int32_t *coords_xyz, int64_t n);

/* Rebuild the block hierarchy from a particle cloud (Sec. 6.3): occupancy of
   level-0 blocks (Phi), the has-children sets H_l (one-block dilation of the
   parents of the finer set), internal blocks (not stored), stored / border /
   leaf sets, flags against the previous hierarchy, stable compaction of the
   stored blocks, neighbour tables and interface node lists.  Blocks that stay
   keep their moments; new fine nodes are interpolated from the coarser level
   (Eq. downward_rescale, spatial part), new coarse nodes take the upward rule
   of Eq. upload_S from their finer coincident nodes.  pos_xyz: float32 [n][3]
   positions in fine-node units, host (on_device = 0, copied) or device
   (on_device = 1, borrowed for the call).  counts_out (host, may be NULL):
   refined (newly in H), coarsened (newly out of H) and deleted blocks summed
   over levels.  Must be called at a coarse-step boundary.  The level-0 force
   field is dropped (set it again for the new block list).  Non-finite
   positions are ignored and reported with HLBM_E_NONFINITE after the rebuild.
   A hierarchy equal to the installed one (no block refined, coarsened,
   deleted or added on any level) keeps the installed levels, lists and
   moments; the interfaces are refilled from the coarser level and the flags
   lose their new / refine / coarsen bits, as a full rebuild would leave them. */
int32_t hlbm_rebuild_from_particles(hlbm_lattice *h, const float *pos_xyz, int64_t n, int32_t on_device,
                                    int64_t counts_out[3]);

/* Per-handle profile: with on != 0, the library records CUDA events on the
   handle's stream around each phase it launches and sums the stream time
   between them per class: 0 stream-collide of every level (coupled steps
   included), 1 downward transfers, 2 upward transfers, 3 open-face updates,
   4 hierarchy rebuilds (whole calls), 5 particle deposits, 6 recordings and
   adjoints (whole calls; they contain classes 0-2), 7 FP64 reductions.
   Off by default; turning it off keeps the totals. */
int32_t hlbm_set_profiling(hlbm_lattice *h, int32_t on);

/* Totals of the profile so far: ms_out[c] (milliseconds of stream time) and
   count_out[c] (spans) for the 8 classes above, host arrays.  Synchronises
   the handle's stream.  reset != 0 zeroes the totals after reading. */
int32_t hlbm_get_profile(hlbm_lattice *h, double ms_out[8], int64_t count_out[8], int32_t reset);

/* Block lookup by position of the rebuilt hierarchies (Sec. 6.1: each
   level's table of active tiles, found through a spatial hash).  mode 0
   (default): a dense slot table per level (int32 per block slot of the
   domain).  mode 1: a spatial hash per level (open addressing, linear
   probing, at most half full: 12 bytes per table entry, 2 to 4 entries per
   stored block); the dense slot table is then dropped after each rebuild.
   The neighbour tables, the interface transfers, the moment carry-over of a
   rebuild, the particle deposit and the multi-level adjoint use whichever is
   present; results are identical.  Takes effect at once for levels already
   built by the rebuild pipeline (a failed allocation leaves them as they
   were) and for every later rebuild.  The rebuild itself still works on
   dense per-level grids.  HLBM_E_INVALID_ARG for another mode. */
int32_t hlbm_set_block_lookup(hlbm_lattice *h, int32_t mode);

/* The block lookup mode and the device bytes the lookup tables of all levels
   hold now (dense slot tables: 4 bytes per block slot of a level; hashes: 12
   bytes per table entry).  Host outputs; HLBM_E_INVALID_ARG for NULL. */
int32_t hlbm_get_block_lookup(const hlbm_lattice *h, int32_t *mode, int64_t *table_bytes);

/* Interface nodes of a level as (block << 9) | node, ascending: which = 0 the
   downward set I^d (filled from level+1 by the downward transfer), which = 1
   the upward set I^u (filled from level-1 by the upward transfer).  Host
   output; if cap < n returns HLBM_E_INVALID_ARG with *n set. */
int32_t hlbm_get_interface_nodes(const hlbm_lattice *h, int32_t level, int32_t which, int32_t *out, int64_t cap,
                                 int64_t *n);

/* Number of stored blocks of a level. */
int32_t hlbm_num_blocks(const hlbm_lattice *h, int32_t level, int64_t *n);

/* Copy the stored block coordinates (bx, by, bz) of a level into out[cap][3]
   (host memory), ascending slot order, and optionally one flag byte per block
   (bit 0 leaf, bit 1 border, bit 2 new, bit 3 refine, bit 4 coarsen; Sec. 6.1,
   Sec. 6.3).  If cap < n, returns HLBM_E_INVALID_ARG with *n set. */
int32_t hlbm_get_blocks(const hlbm_lattice *h, int32_t level, int32_t *out, int64_t cap,
                        int64_t *n, uint8_t *flags_out);

/* Coupling fields of the finest level from a particle cloud (Sec. 4: the
   solid fraction eta enters through eps = 1 - eta and the force F).  Per
   finest-level node: count(x) = particles whose floor(position) is x (clamped
   to the domain), eta = min(eta_max, per_particle * count), eps = 1 - eta and
   F = (0, -kappa * eta, 0) if moving, else 0; FP64 arithmetic rounded once to
   float32.  Replaces the level-0 force and eps fields (like hlbm_set_force).
   pos_xyz: float32 [n][3] in fine-node units, host (on_device = 0) or device
   (1, borrowed until the call's work on the stream has run).  Particles that
   fall in no stored finest-level block or are not finite are dropped; with
   outside != NULL the call waits for the stream and stores their number in
   *outside (host), with outside == NULL it returns without waiting. */
int32_t hlbm_deposit_particles(hlbm_lattice *h, const float *pos_xyz, int64_t n, int32_t on_device, double kappa,
                               double eta_max, double per_particle, int32_t moving, int64_t *outside);

/* Uniform body force F (lattice units) at level 0 (Sec. 4, force F). */
int32_t hlbm_set_uniform_force(hlbm_lattice *h, double fx, double fy, double fz);

/* Per-node force F[n_blocks0][3][512] and fluid fraction eps[n_blocks0][512]
   (float32, device memory, level-0 block order) for the forcing and the mixture
   relaxation time eps*tau of Sec. 4.  Copied device-to-device; eps may be NULL
   (eps = 1).  F may be NULL to return to the uniform force.  A non-finite
   value in either buffer returns HLBM_E_NONFINITE and changes nothing
   (synchronous check). */
int32_t hlbm_set_force(hlbm_lattice *h, const float *F_dev, const float *eps_dev);

/* Live drag of the coupled LBM step (Fig. 4, Sec. 5.4: streaming only, force
   exchange, then collision).  With exchange_every = k > 0, every k-th level-0
   step from now on (the first one included) streams, computes the drag
     F = kappa * (1 - eps) * (vp - u*),  u* = j* / rho*
   at every level-0 node from the streamed (pre-collision) moments, the fluid
   fraction eps of the last hlbm_set_force / hlbm_deposit_particles (1 if
   none) and the sediment velocity vp[3] (lattice units, host), stores it as
   the level-0 force field (as hlbm_set_force would) and collides with it; the
   steps in between use that field unchanged.  exchange_every = 0 turns the
   exchange off (the field stays).  kappa and vp must be finite
   (HLBM_E_INVALID_ARG); FP64 storage is refused (HLBM_E_UNSUPPORTED); while
   the drag is on, hlbm_forward_record is refused (the adjoint takes F as
   fixed).  Each exchange step holds one float32 moment-sized buffer of the
   finest level (40 B per node) while it runs. */
int32_t hlbm_set_drag(hlbm_lattice *h, double kappa, const double vp[3], int32_t exchange_every);

/* Open faces (the open scenes of Sec. 7): type[6] for the faces x-, x+, y-,
   y+, z-, z+ (hlbm_face), host memory.  An open face needs a non-periodic
   axis (it replaces the wall there).  The nodes of an open face layer keep
   their moments in the step of their level; after every step of every level
   they are written from the state before the step:
   - HLBM_FACE_OUTFLOW: the convective equation dM/dt + u_n dM/dn = 0, first
     order upwind: M_b <- M_b - c (M_b - M_i), with M_i the node one step
     inward and c = clamp(u_n, 0, 1) its velocity along the outward normal
     (the paper takes u_n from the nearest interior node);
   - HLBM_FACE_INLET: density of M_i, velocity u(h) = u0 ln(1 + beta (h - h0))
     along the inward normal (0 where 1 + beta (h - h0) <= 1), S = u u; h is
     the node's coordinate along profile_axis in finest-level node units.
   A node on several open faces takes the first open face in the order above.
   HLBM_E_INVALID_ARG for an unknown type, an open face on a periodic axis, a
   profile axis equal to an inlet face's axis or non-finite inlet values.
   The adjoint is refused while a face is open.  May be called before or after
   the blocks are set; the neighbour tables and bounce masks are rebuilt. */
int32_t hlbm_set_open_faces(hlbm_lattice *h, const int32_t type[6], double u0, double beta, double h0,
                            int32_t profile_axis);

/* Solid nodes of a single-level lattice, one byte per fine node (host memory,
   dense [nz][ny][nx], non-zero = solid).  Solid nodes are frozen at rest and
   fluid nodes next to them use half-way bounce-back.  NULL clears. */
int32_t hlbm_set_solid(hlbm_lattice *h, const uint8_t *mask_dense);

/* Write / read the stored moments of a level, block-major [n][10][512].
   dtype 0 = float64, 1 = float32.  on_device 0 = host pointer, 1 = device
   pointer.  For reads, physical_u = 1 returns u = u' - F/(2 rho) at level 0.
   A write whose buffer holds a non-finite value returns HLBM_E_NONFINITE and
   leaves the level unchanged (the check waits for the stream).  A state that
   turns non-finite while stepping is reported by hlbm_reduce. */
int32_t hlbm_write_moments(hlbm_lattice *h, int32_t level, const void *buf, int32_t dtype,
                           int32_t on_device);
int32_t hlbm_read_moments(hlbm_lattice *h, int32_t level, void *buf, int32_t dtype,
                          int32_t on_device, int32_t physical_u);

/* Advance n_fine_steps finest-level steps (Algorithm 1 called
   n_fine_steps / 2^(L-1) times); n_fine_steps must be a multiple of 2^(L-1).
   Asynchronous on the handle's stream. */
int32_t hlbm_step(hlbm_lattice *h, int32_t n_fine_steps);

/* Wait for the handle's stream. */
int32_t hlbm_synchronize(hlbm_lattice *h);

/* FP64 reductions over nodes not covered by a finer level, weighted by the
   cell volume 8^l: out[0] mass, out[1..3] momentum (physical u), out[4]
   kinetic energy, out[5] mass at level 0, out[6] mass at the other levels.
   Synchronous.  Returns HLBM_E_NONFINITE if the mass is not finite. */
int32_t hlbm_reduce(hlbm_lattice *h, double out[7]);

/* Reverse mode of the stream-collide step (the paper has no adjoint; this
   differentiates Sec. 3.1 with the Guo force and eps*tau of Sec. 4 with
   respect to the level-0 force field) and, on lattices whose blocks come from
   the rebuild pipeline (hlbm_set_fine_blocks / hlbm_rebuild_from_particles),
   of the whole multi-level advance of Algorithm 1: sub-cycled level steps,
   the downward transfer with its temporal midpoint and the upward transfer,
   both with their S^neq rescaling (Sec. 5.2, 5.3).
   hlbm_forward_record advances n_steps fine steps like hlbm_step and keeps
   the state every ckpt_every fine steps (device memory; multi-level: every
   level's current state, and both counts must be multiples of 2^(L-1)).
   hlbm_adjoint then takes dL/dM of the final stored moments (float32 device
   buffer, public layout [nb][10][512], rho row = d/d rho; multi-level: every
   level's blocks in level order, level 0 first) and writes dL/dF (float32
   device [nb0][3][512], the layout of hlbm_set_force) by recomputing each
   checkpoint segment and stepping backwards; the force sums are FP64.  With
   FP32 storage hlbm_forward_record runs its last segment the way the adjoint
   recomputes one and keeps it (the tape), so hlbm_adjoint recomputes every
   segment but that one; the tape's buffers are the segment buffers listed
   below, allocated by hlbm_forward_record and held until the next
   hlbm_adjoint, which takes them over and frees them (a further hlbm_adjoint
   on the same recording recomputes every segment).
   Device memory of the segment buffers, single level: with FP32 storage, the K =
   ckpt_every states and pre-collision moment fields of one segment (2 K x 40
   B per node) plus four float32 moment-sized buffers and the FP64 dL/dF sum
   (24 B per node); with FP64 storage, K - 1 states (80 B per node each) and
   the same buffers.  Multi-level: per level step of a segment one state and
   one pre-collision field (2 x 40 B per node of that level), the values each
   transfer overwrites, one working copy of the checkpoint, and 2 L + 2
   float32 moment-sized buffers of the largest level.
   Single-level lattices with FP32 or FP64 storage, multi-level lattices with
   FP32 storage (HLBM_E_UNSUPPORTED otherwise); force, eps and solids must not
   change between the two calls, and a change of the block layout in between
   makes hlbm_adjoint fail with HLBM_E_BAD_STATE.  Synchronous. */
int32_t hlbm_forward_record(hlbm_lattice *h, int32_t n_steps, int32_t ckpt_every);
int32_t hlbm_adjoint(hlbm_lattice *h, const float *dL_dM_dev, float *dL_dF_dev);

/* Test hook for the error paths: after `after` more successful device
   allocations (by any lattice or batch handle), the next one fails and its call returns
   HLBM_E_OOM, as a real out-of-memory would; later allocations succeed
   again.  after < 0 clears a pending failure.  Always returns HLBM_OK.
   After a failed allocation the handle stays safe to use and to destroy:
   a failed rebuild (hlbm_set_fine_blocks / hlbm_rebuild_from_particles)
   keeps the previous hierarchy and state; a failed hlbm_set_dense leaves
   no blocks (HLBM_E_BAD_STATE until blocks are set again); a failed
   hlbm_set_force or hlbm_deposit_particles keeps the previous fields; a
   failed hlbm_forward_record or hlbm_adjoint frees its buffers and records
   nothing; a failed coupled step leaves the moments of that step
   undefined. */
int32_t hlbm_inject_alloc_failure(int64_t after);

/* Test hook: writes to out_dev[i] the binary64 -> binary32 round-to-nearest-
   even narrowing that the interface transfers apply to their FP64 sums
   (integer arithmetic for results in the normal binary32 range), and to
   hw_dev[i] the CUDA conversion instruction's result, for n device values
   in_dev.  Synchronous; HLBM_E_INVALID_ARG for n < 0 or NULL buffers with
   n > 0. */
int32_t hlbm_test_narrow(const double *in_dev, float *out_dev, float *hw_dev, int64_t n);

/* Allocation-free FP64 reduction of a moment buffer the caller already holds.
 * The paper has no counterpart; this entry point exists for callers that must
 * not allocate device memory: code embedded in a host application that owns
 * the allocator (a plugin inside another solver), loops with a fixed memory
 * budget, or contexts where allocation would synchronise the device.
 *
 * mom_dev:  float32 device buffer in the public layout [n_blocks][10][512]
 *           (rho in row 0), as written by hlbm_read_moments with on_device = 1
 *           and physical_u = 0: the velocity rows must hold the stored
 *           velocity u' = u + F/(2 rho), since this call subtracts F/(2 rho)
 *           itself (a buffer read with physical_u = 1 would be shifted twice).
 *           Every node of every block is summed with unit volume: the result
 *           equals hlbm_reduce for single-level lattices only (hlbm_reduce
 *           leaves out blocks covered by a finer level and weights level l
 *           by 8^l).
 * F_dev:    float32 device force [n_blocks][3][512], or NULL to use (fx, fy, fz);
 *           the velocity summed is u' - F/(2 rho).
 * out_dev:  five doubles in device memory, overwritten with mass, momentum
 *           (3) and kinetic energy.
 * stream:   cudaStream_t (NULL = legacy default stream); the call is
 *           asynchronous on it.
 * Scratch:  a fixed file-scope device array sized for at most 65,536 blocks
 *           (3.7 MB, present on every GPU that loads the library until the
 *           process exits).  n_blocks outside [1, 65536] returns
 *           HLBM_E_INVALID_ARG (message in hlbm_last_error(NULL)).  No
 *           allocation or free is made by this call.  The first call on a
 *           device looks up the scratch address with that device current, so
 *           make that first call outside any stream capture.  All calls share
 *           the one scratch array: calls whose kernels overlap on the GPU race
 *           and must be serialised (one stream, or events). */
int32_t hlbm_reduce_f32_noalloc(const float *mom_dev, int64_t n_blocks, const float *F_dev, double fx, double fy,
                                double fz, double *out_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Batches of independent domains.  The paper runs one lattice at a time; a
 * batch advances many small single-level periodic domains (8^3 blocks, FP32,
 * FP16S or BF16S storage, each its own extent and tau) with one kernel launch
 * per step over the concatenated block list, so that small domains fill the
 * GPU together.  Each domain keeps its own reduced-precision row scales.
 * ------------------------------------------------------------------------- */
typedef struct hlbm_batch hlbm_batch;

typedef enum {
  HLBM_BATCH_ONE_LAUNCH = 0, /* one launch per step over every domain */
  HLBM_BATCH_GRAPH = 1,      /* the same, 32 steps at a time replayed from a CUDA graph (default) */
  HLBM_BATCH_PER_DOMAIN = 2, /* one launch per domain per step (for comparison) */
  HLBM_BATCH_PERSISTENT = 3, /* one launch per step of resident CTAs taking blocks from an atomic counter */
  HLBM_BATCH_PERSISTENT_GRAPH = 4 /* the same, 32 steps at a time from a CUDA graph */
} hlbm_batch_mode;

/* Create a batch of n domains from cfgs[n]: every domain single-level, fully
   periodic, block_edge 8, extents multiples of 8; storage, device and stream
   equal across domains (a NULL stream makes the batch create its own, since
   CUDA graphs cannot capture the legacy stream).  Moments start at rest.
   *out is NULL on failure (message in hlbm_batch_last_error(NULL)). */
int32_t hlbm_batch_create(const hlbm_config *cfgs, int32_t n, hlbm_batch **out);
/* Free the batch.  NULL is accepted. */
int32_t hlbm_batch_destroy(hlbm_batch *b);
/* Message of the last failed call on b (NULL: of the last failed create). */
const char *hlbm_batch_last_error(const hlbm_batch *b);
/* Blocks of one domain (domain = -1: of the whole batch).  A domain's blocks
   are in x-fastest block order, like hlbm_get_blocks of a dense lattice. */
int32_t hlbm_batch_num_blocks(const hlbm_batch *b, int32_t domain, int64_t *n);
/* Write / read one domain's moments in the public layout [n][10][512]
   (dtype 0 = float64, 1 = float32; host or device pointer).  Synchronous.
   Writing refits that domain's row scales (reduced-precision storage). */
int32_t hlbm_batch_write_moments(hlbm_batch *b, int32_t domain, const void *buf, int32_t dtype, int32_t on_device);
int32_t hlbm_batch_read_moments(hlbm_batch *b, int32_t domain, void *buf, int32_t dtype, int32_t on_device);
/* Advance every domain n_steps steps (Sec. 3.1 with zero force), asynchronous
   on the batch's stream; reduced-precision scales are refit every 32 steps.
   Results do not depend on the mode. */
int32_t hlbm_batch_step(hlbm_batch *b, int32_t n_steps);
int32_t hlbm_batch_synchronize(hlbm_batch *b);
/* Choose the launch strategy (hlbm_batch_mode). */
int32_t hlbm_batch_set_mode(hlbm_batch *b, int32_t mode);
/* Time each mode over trial_steps steps (at least 64; the state is restored
   afterwards), keep the fastest and return it in *mode_out; ms_out (host, may
   be NULL) receives the five per-step times in mode order.  Synchronous. */
int32_t hlbm_batch_autotune(hlbm_batch *b, int32_t trial_steps, int32_t *mode_out, float ms_out[5]);

#ifdef __cplusplus
}
#endif
#endif /* HOMELBM_H */
