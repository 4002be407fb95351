/*
 * lbm.h - C ABI of the GB300-native disaggregated D3Q19 lattice-Boltzmann
 * library (liblbm.so).
 *
 * The library implements the fused stream-and-collide D3Q19 update of the
 * paper "Disaggregated Design for GPU-Based Volumetric Data Structures"
 * (Sec. 6: LBM with BGK collision, D3Q19; Sec. 6.2: bounce-back and
 * regularized inflow/outflow boundaries) over the paper's disaggregated
 * layouts: voxels are first grouped by a trait (Sec. 2, Definition:
 * definition / classification / mapping / operations) and then laid out
 * for locality inside each group:
 *   - dense grids (Sec. 3): boundary-trait voxels form their own contiguous
 *     SoA group, processed by their own kernel;
 *   - block-sparse grids (Sec. 4, Table 2 "Disag - Mem"): boundary blocks are
 *     stored first, non-boundary blocks after, one lean kernel per group;
 *   - multi-resolution grids (Sec. 5, Sec. 6.3): per level, blocks next to a
 *     resolution jump (G_c) are separated from uniform blocks (G_i), which
 *     run fused at every level.
 *
 * Conventions shared by every call
 *   - All functions return lbm_status; they never abort or trap.  On error,
 *     lbm_last_error() returns a thread-local message.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Host arrays passed in are only read during the call and stay owned by
 *     the caller.  Device memory of a grid is owned by the library and is
 *     obtained through the lbm_allocator given at creation (NULL allocator:
 *     cudaMalloc / cudaFree).  Output buffers belong to the caller.
 *   - Virtual-box arrays are indexed x fastest: v = x + nx*(y + ny*z).
 *   - Flag byte per voxel: bits 0-2 type (0 fluid, 1 solid / bounce-back,
 *     2 regularized velocity node, 3 regularized pressure node, 7 not in
 *     domain); bits 3-5 outward normal index of a regularized node
 *     (0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z).
 *   - Lattice: D3Q19, velocities ordered rest, +x, -x, +y, -y, +z, -z,
 *     (+1,+1,0), (-1,-1,0), (+1,-1,0), (-1,+1,0), (+1,0,+1), (-1,0,-1),
 *     (+1,0,-1), (-1,0,+1), (0,+1,+1), (0,-1,-1), (0,+1,-1), (0,-1,+1).
 *   - Stored state: post-collision populations f* (pull scheme).
 *   - Asynchronous device errors are latched in a per-grid status word and
 *     reported by the next lbm_sync / lbm_get_* call.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_grid lbm_grid;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_INVALID = 1,     /* bad argument or descriptor                      */
  LBM_ERR_OOM = 2,         /* allocation failed (nothing leaked)              */
  LBM_ERR_CUDA = 3,        /* a CUDA runtime call failed                      */
  LBM_ERR_TIMEOUT = 4,     /* a bounded device wait ran out                   */
  LBM_ERR_DIVERGED = 5,    /* non-finite mass / momentum                      */
  LBM_ERR_UNSUPPORTED = 6, /* valid request the library does not implement   */
  LBM_ERR_INTERNAL = 7     /* library invariant broken (device-side check)    */
} lbm_status;

enum { LBM_COLLISION_BGK = 0, LBM_COLLISION_REG = 1 };
enum { LBM_STORAGE_F32 = 0, LBM_STORAGE_F16 = 1, LBM_STORAGE_BF16 = 2 };
/* Kernel schedule.  DISAGGREGATED: one lean kernel per voxel group (the
 * paper's design; on block-sparse grids its memory-based grouping, Sec. 4:
 * boundary blocks stored first, then the rest, each kernel over its own
 * contiguous range).  MONOLITHIC: one kernel with per-voxel branches over every
 * voxel (the paper's "naive" kernel, Sec. 4 and Table 2); for multi-resolution
 * grids it selects the unfused collide / stream pair on every block (the
 * baseline of Sec. 6.3).  BITMASK (block-sparse grids only, chosen at
 * creation): the bitmask-based grouping of Sec. 4 and Table 2 — every block
 * in Morton order whatever its group, a per-block bit marks the boundary
 * blocks, both group kernels run over all blocks and skip the other group's,
 * and boundary values are reached through a per-slot index into a compact
 * buffer (indirect indexing).  A grid created with BITMASK may switch only
 * to MONOLITHIC and back; a grid created otherwise cannot switch to BITMASK
 * (LBM_ERR_UNSUPPORTED): the block order is fixed at creation. */
enum { LBM_SCHEDULE_DISAGGREGATED = 0, LBM_SCHEDULE_MONOLITHIC = 1, LBM_SCHEDULE_BITMASK = 2 };

typedef struct {
  double tau;        /* BGK relaxation time of the finest level, > 0.5        */
  int collision;     /* LBM_COLLISION_*                                       */
  int storage;       /* LBM_STORAGE_*; F16 / BF16 store f_i - w_i (RN-even)   */
  int closure;       /* 0 none, 1 learned tau correction (multi-res levels)   */
  int periodic[3];   /* per axis: 1 periodic, 0 bounce-back walls at the box  */
  int schedule;      /* LBM_SCHEDULE_*                                        */
  int lattice;       /* 19 (D3Q19) or 27 (D3Q27); 0 means 19.  D3Q27 runs on
                        dense, block-sparse and multi-resolution grids (every
                        schedule, both collisions, all storages, regularized
                        boundaries); the closure and batches are D3Q19
                        (LBM_ERR_UNSUPPORTED otherwise).  Populations
                        are indexed i = 0..Q-1 in the order: rest, the six
                        axis directions, the twelve edge directions (D3Q19's
                        order), then (D3Q27) the eight corners (+1,+1,+1),
                        (-1,-1,-1), (+1,+1,-1), (-1,-1,+1), (+1,-1,+1),
                        (-1,+1,-1), (-1,+1,+1), (+1,-1,-1)                    */
} lbm_physics;

typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream); /* NULL on failure */
  void (*free)(void* ctx, void* p, void* stream);
} lbm_allocator;

typedef struct {
  int kind;                 /* 0 dense, 1 sparse, 2 multi-resolution          */
  int n_levels;
  int dims[3];              /* virtual box of level 0                         */
  int block_edge;           /* sparse / multi-res block edge (0 for dense)    */
  int64_t n_updated[4];     /* updated voxels per level (fluid + regularized) */
  int64_t n_blocks[4];      /* active blocks per level                        */
  int64_t n_group_b[4];     /* boundary blocks (sparse) / G_c blocks (multi)  */
  int64_t n_regularized;    /* regularized voxels (all levels)                */
  size_t population_bytes[4]; /* bytes of one population buffer per level     */
  int64_t steps_done;
  int lattice;              /* 19 or 27                                       */
} lbm_info;

/* ---------------------------------------------------------------- grids */

/* Dense grid of dims[0] x dims[1] x dims[2] voxels, all fluid until
 * lbm_set_boundary.  Storage: one SoA array per population, index
 * pop * N + v (Sec. 3, SoA; Sec. 6.1 dense LBM). */
lbm_status lbm_grid_create_dense(const int dims[3], const lbm_physics* phys,
                                 const lbm_allocator* alloc, void* stream,
                                 lbm_grid** out);

/* Block-sparse grid (Sec. 4; Sec. 6.2).  `flags` (host, virtual box) fixes
 * the active blocks (a block is active iff it holds a voxel of type 0, 2 or 3)
 * and the groups: a block is a boundary block iff it holds a regularized
 * voxel (Sec. 6.2).  Numbering: boundary blocks first, then non-boundary
 * blocks, each in ascending Morton order of the block coordinate (x lowest
 * bit).  Storage index ((block * Q) + pop) * E^3 + lx + E*(ly + E*lz), Q = 19
 * or 27 (phys->lattice).
 * block_edge must be 4 or 8; periodic axes need dims divisible by it. */
lbm_status lbm_grid_create_sparse(const int dims[3], int block_edge,
                                  const uint8_t* flags, const lbm_physics* phys,
                                  const lbm_allocator* alloc, void* stream,
                                  lbm_grid** out);

/* Multi-resolution grid (Sec. 5; Sec. 6.3), refinement factor 2, level 0 =
 * finest, 1 <= n_levels <= 4.  Axes may be periodic or walled
 * (phys->periodic); walls, solids and regularized voxels lie on level 0
 * only (lbm_set_boundary on level 0), so every map cell touching a walled
 * box side must belong to level 0 (LBM_ERR_UNSUPPORTED otherwise) — the
 * lid-driven cavity of Sec. 6.3 / Table 5 has its finest level along the
 * walls.  level_map (host) gives the owning level of every cube of
 * C = 8 * 2^(n_levels-1) finest voxels, indexed x fastest over
 * finest_dims / C cells; finest_dims must be multiples of C and neighbouring
 * cells (26-neighbourhood, periodic) may differ by at most one level.
 * Each level is an 8^3-block sparse grid in its own voxel units; per level,
 * blocks with a D3Q19 neighbour on another level (G_c) are numbered first,
 * then the others (G_i), each in Morton order.  Level l relaxes with
 * tau_l = 1/2 + (tau - 1/2) / 2^l (acoustic scaling, one viscosity) and
 * advances 2^(n_levels-1-l) times per lbm_step step. */
lbm_status lbm_grid_create_multires(const int finest_dims[3], int n_levels,
                                    const uint8_t* level_map, const lbm_physics* phys,
                                    const lbm_allocator* alloc, void* stream,
                                    lbm_grid** out);

lbm_status lbm_grid_destroy(lbm_grid* g);

lbm_status lbm_get_info(const lbm_grid* g, lbm_info* out);

/* Select the kernel schedule (LBM_SCHEDULE_*) for later lbm_step calls. */
lbm_status lbm_set_schedule(lbm_grid* g, int schedule);

/* Interior-kernel variant of a dense grid (no counterpart in the paper; a
 * tuning knob of this implementation):
 *   LBM_VARIANT_VEC16  a thread moves 16-byte vectors of consecutive voxels,
 *   LBM_VARIANT_SCALAR one voxel per thread (default),
 *   LBM_VARIANT_VEC8   8-byte vectors,
 *   LBM_VARIANT_VEC4   4-byte vectors (two voxels per thread under FP16 /
 *                      BF16 storage; the scalar kernel under FP32).
 * Vector variants apply when walls are only box sides, dims[0] is a multiple
 * of the vector length and the boundary group is whole top planes; otherwise
 * the scalar kernel runs.  Block-sparse and multi-resolution grids with 8^3
 * blocks take LBM_VARIANT_STAGED: the lean kernel copies each block's
 * populations to shared memory with one bulk asynchronous copy (the tensor
 * memory accelerator, completion on an mbarrier) and pulls the in-block
 * sources from there, the cross-block ones from global memory; any other
 * value selects their default kernel (LBM_ERR_UNSUPPORTED for a dense grid
 * or 4^3 blocks).  Results are identical across variants. */
enum { LBM_VARIANT_VEC16 = 0, LBM_VARIANT_SCALAR = 1, LBM_VARIANT_VEC8 = 2, LBM_VARIANT_VEC4 = 3,
       LBM_VARIANT_STAGED = 4 };
lbm_status lbm_set_variant(lbm_grid* g, int variant);

/* Time limit of the staged kernel's wait (LBM_VARIANT_STAGED; no counterpart
 * in the paper).  Each CTA of that kernel waits for the bulk copy of its
 * block on an mbarrier for at most `ns` nanoseconds of the GPU's global
 * timer (default 200 ms; ns < 0 restores it).  A CTA whose wait runs out
 * updates nothing, latches LBM_ERR_TIMEOUT (reported by lbm_sync) and, before
 * it exits, drains its copy for up to one second more, so no copy can land
 * in shared memory the CTA has released.  ns = 0 makes every wait run out at
 * once, which is how the timeout path is tested; the state of that step is
 * then not a valid update. */
lbm_status lbm_set_wait_limit(lbm_grid* g, int64_t ns);

/* Autotuner: times each variant that applies to the grid (the four dense
 * interior variants; LBM_VARIANT_SCALAR and LBM_VARIANT_STAGED on 8^3-block
 * sparse and multi-resolution grids) over n_steps steps (CUDA events on the
 * grid's stream) starting from the grid's current state, restores that state,
 * and keeps the fastest.  *chosen receives it; ms_per_step (5 doubles, one
 * per LBM_VARIANT_*, 0 for a variant not timed, or NULL) receives the
 * measured time per step of each. */
lbm_status lbm_autotune(lbm_grid* g, int n_steps, int* chosen, double* ms_per_step);

/* Voxel types and boundary values of one level.
 *   flags     host virtual box, or NULL to keep the current flags.  On a
 *             sparse grid non-NULL flags must equal the creation flags.
 *   bc_values host, 4 floats (ux, uy, uz, rho) per regularized voxel in
 *             flag-scan order (x fastest), or NULL to use default_bc for all.
 *   default_bc 4 floats, used when bc_values is NULL (may be NULL when there
 *             are no regularized voxels).
 * Velocity nodes use (ux, uy, uz); pressure nodes use rho (Sec. 6.2 inflow /
 * outflow).  Dense grids re-derive their groups here: regularized voxels form
 * the boundary group; when they are the last voxels in memory (a top lid) the
 * interior kernel covers the rest as one contiguous range. */
lbm_status lbm_set_boundary(lbm_grid* g, int level, const uint8_t* flags,
                            const float* bc_values, const float default_bc[4]);

/* Initial state f* = f^eq(rho, u), evaluated in FP64 on the GPU and stored in
 * the grid's storage format.  The stored state of the pull scheme is the
 * post-collision population f* (Sec. 6: collide and stream fused in one
 * kernel), and f^eq is the second-order equilibrium of the BGK model the
 * paper names (Sec. 6), w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u).  rho: n doubles (NULL -> 1); u: 3*n doubles,
 * component-major (ux[n], uy[n], uz[n]) (NULL -> 0); n = level's virtual box
 * voxel count.  device_ptrs: 0 host arrays, 1 device arrays.  Page-locked
 * host arrays mapped into the device address space are read by the kernel
 * in place; other host arrays are staged through device scratch.  Voxels
 * that are not updated are ignored. */
lbm_status lbm_init_equilibrium(lbm_grid* g, int level, const double* rho,
                                const double* u, int device_ptrs);

/* Advance n_steps time steps (coarsest steps on a multi-resolution grid) on
 * `stream`.  One step is the fused stream-and-collide update of Sec. 6 (pull
 * g_i(x) = f*_i(x - c_i), halfway bounce-back on walls and obstacles and the
 * regularized inflow / outflow nodes of Sec. 6.2, BGK or regularized
 * collision), run as one lean kernel per voxel group (Sec. 2 Definition;
 * Sec. 3 dense, Sec. 4 / Table 2 block-sparse); on a multi-resolution grid
 * level l advances 2^(n_levels-1-l) times with explosion / coalescence at the
 * level jumps and fused uniform blocks on every level (Sec. 5, Sec. 6.3).  Asynchronous; device errors are latched.  The steps order after
 * the grid's work on the stream of its previous call (and on `stream`); the
 * other calls then use `stream`.  LBM_ERR_INVALID when the grid has
 * regularized voxels whose boundary values were never given
 * (lbm_set_boundary). */
lbm_status lbm_step(lbm_grid* g, int n_steps, void* stream);

/* Density and velocity of the stored state in FP64, virtual-box order, NaN on
 * voxels that are not updated: rho = sum_i f*_i, u = sum_i f*_i c_i / rho,
 * the macroscopic moments of the LBM state (Sec. 6).  rho: n doubles or NULL; u: 3*n doubles
 * (component-major) or NULL.  Page-locked, mapped host arrays are written by
 * the kernel in place.  Synchronises the grid's stream. */
lbm_status lbm_get_moments(lbm_grid* g, int level, double* rho, double* u,
                           int device_ptrs);

/* Raw stored populations (checkpoint format = the grid's storage layout and
 * precision): the dense SoA arrays of Sec. 3 (pop * N + v) or the per-block
 * arrays of Sec. 4 ((block * Q + pop) * E^3 + voxel), post-collision f*.
 * bytes must equal info.population_bytes[level]. */
lbm_status lbm_get_populations(lbm_grid* g, int level, void* dst, size_t bytes,
                               int device_ptrs);
lbm_status lbm_set_populations(lbm_grid* g, int level, const void* src,
                               size_t bytes, int device_ptrs);

/* Stored populations decoded to FP64 in virtual-box order:
 * dst[pop * n + v], NaN on voxels that are not updated. */
lbm_status lbm_get_populations_f64(lbm_grid* g, int level, double* dst,
                                   int device_ptrs);

enum {
  LBM_LAYOUT_FLAGS = 0,        /* uint8  virtual box                           */
  LBM_LAYOUT_BLOCK_COORDS = 1, /* int32  n_blocks x 3 (bx, by, bz)             */
  LBM_LAYOUT_NBR = 2,          /* int32  n_blocks x 27, -1 = none              */
  LBM_LAYOUT_BLOCK_MAP = 3,    /* int32  virtual block grid -> block id or -1  */
  LBM_LAYOUT_XNBR_COARSE = 4,  /* int32  n_blocks x 27 (multi-res)             */
  LBM_LAYOUT_XNBR_FINE = 5,    /* int32  n_blocks x 27 x 8 (multi-res)         */
  LBM_LAYOUT_BOUNDARY_BITS = 6,/* uint32 ceil(n_blocks / 32): bit b % 32 of word
                                  b / 32 = block b is a boundary block (BITMASK) */
  LBM_LAYOUT_BC_INDEX = 7,     /* int32  n_blocks x E^3: rank of the slot's
                                  regularized voxel in flag-scan order, or -1
                                  (BITMASK)                                     */
  LBM_LAYOUT_IFACE_SLOTS = 8,  /* int32  n_iface: slots (block * 512 + voxel) of
                                  the level's interface voxels, ascending: the
                                  voxels with a pull whose value depends on
                                  another level (multi-res; Sec. 5, P_d = 0) */
  LBM_LAYOUT_IFACE_CROSS = 9   /* uint32 n_iface: bit i = population i of that
                                  voxel comes from explosion (from the coarser
                                  level) or coalescence (from the finer one)  */
};
/* Copy one host-side layout table (for bit-exact checks).  bytes must equal
 * the table's size; lbm_layout_bytes reports it. */
lbm_status lbm_layout_bytes(const lbm_grid* g, int level, int what, size_t* bytes);
lbm_status lbm_get_layout(const lbm_grid* g, int level, int what, void* dst,
                          size_t bytes);

/* Conservation sums over every updated voxel of every level, accumulated in
 * FP64 on the GPU with a deterministic two-pass warp-shuffle reduction:
 * out[0] = sum_l 8^l sum f*_i, out[1..3] = sum_l 8^l sum f*_i c_i.
 * Returns LBM_ERR_DIVERGED when a sum is not finite.  Synchronises. */
lbm_status lbm_conservation(lbm_grid* g, double out_mass_mom[4]);

/* Conservation sums of a dense population buffer without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate at the point they need the sums, e.g. a solver
 * loop that must not synchronise the device (cudaMalloc / cudaFree may wait
 * for all outstanding work) or an application whose device memory belongs to
 * its own pool.
 *   f            device, dense SoA populations f[pop * n_voxels + v], Q
 *                arrays of the given lattice (the layout of a dense grid's
 *                lbm_get_populations) in the given storage (LBM_STORAGE_*;
 *                F16 / BF16 hold f_i - w_i, w_i that lattice's weights)
 *   lattice      19 (D3Q19) or 27 (D3Q27); 0 means 19
 *   flags        device, one flag byte per voxel, or NULL (all fluid); only
 *                voxels of type 0, 2 and 3 are summed
 *   out_mass_mom device, 4 doubles: sum f_i, sum f_i c_i (FP64, deterministic)
 * f, flags and out_mass_mom must be device (or managed) memory of the current
 * device: host or unregistered pointers return LBM_ERR_INVALID before any
 * launch (checked with cudaPointerGetAttributes, which neither allocates nor
 * synchronises); the buffer sizes cannot be checked and are the caller's.
 * Asynchronous on `stream`; no allocation, copy or synchronisation.  The
 * partial sums live in one fixed device array of 4096 x 4 doubles per device
 * (held until the process exits), so n_voxels <= 67,108,864; larger inputs
 * return LBM_ERR_INVALID.  The first successful call on each device looks up
 * that array's device address (cudaGetSymbolAddress, with that device
 * current; a failed lookup is retried by the next call); make that first call
 * before any stream capture.  Calls share the array: calls that overlap on
 * the GPU race, so order them on one stream. */
lbm_status lbm_conservation_noalloc(const void* f, int storage, int lattice, int64_t n_voxels,
                                    const uint8_t* flags, double* out_mass_mom, void* stream);

/* ------------------------------------------------------- learned closure
 * Not in the paper (the learned part of this implementation): a per-voxel
 * network 16 -> 64 (ReLU) -> 64 (ReLU) -> 1 predicts a relaxation-time
 * correction d_tau on multi-resolution levels >= 1; those voxels relax with
 * tau_eff = max(tau_l + d_tau, 1/2 + 1e-3).  Features per voxel, from the
 * pulled populations g (d = g - f^eq):  rho - 1, u (3), Pi^neq (xx, yy, zz,
 * xy, xz, yz) / (rho/3), |Pi^neq|_F / (rho/3), tr Pi^neq / (rho/3),
 * q_x, q_y, q_z / (rho/3) with q_x = sum_i c_ix (c_iy^2 + c_iz^2) d_i and
 * cyclic, tau_l.  Parameters: 5313 FP32 values, W1 (64 x 16, row per unit),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1).  Inference runs inside the
 * collision kernels as BF16 tensor-core MMAs (weights rounded to BF16, biases
 * FP32, FP32 accumulation). */

/* Training data made by the solver from a dense periodic grid's current
 * state: the state is box-filtered by r^3 (mean populations), streamed one
 * coarse step, and turned into 16 features per coarse voxel; the target is
 * the least-squares eddy viscosity over each coarse voxel's 3^3 neighbourhood,
 * d_tau = -3 sum(tau_sgs_dev : S) / sum(2 rho S : S), clamped to
 * [-(tau_coarse - 1/2) + 1e-3, 1/2].  feats (n_c x 16) and targets (n_c) are
 * device arrays, n_c = voxels / r^3 in coarse x-fastest order.  Synchronises. */
lbm_status lbm_closure_dataset(lbm_grid* fine, int r, double tau_coarse, float* feats,
                               float* targets);

/* Train the network on device arrays feats (n x 16) and targets (n) with
 * MSE loss and Adam (beta 0.9 / 0.999, eps 1e-8, learning rate lr) for
 * `steps` minibatches of `batch` samples drawn by SplitMix64 on counter
 * step*batch + b plus `seed`.  Features and targets are standardised
 * internally (mean and population standard deviation of each column; a
 * column whose deviation is below 1e-6 of its mean's magnitude counts as
 * constant and keeps scale 1); theta_io (device, 5313 FP32) holds the initial weights for the
 * standardised problem and receives the trained weights with the
 * standardisation folded in (they take raw features).  loss_out (host, may
 * be NULL) receives the last minibatch loss (standardised).  Synchronises. */
lbm_status lbm_closure_train(const float* feats, const float* targets, int64_t n, int steps,
                             int batch, float lr, uint64_t seed, float* theta_io,
                             float* loss_out, void* stream);

/* Loss (MSE) and gradient (5313 FP32) of one minibatch, samples idx[0..batch),
 * at weights theta, in FP32; all device pointers.  Synchronises. */
lbm_status lbm_closure_grad(const float* theta, const float* feats, const float* targets,
                            const int32_t* idx, int batch, float* grad, float* loss,
                            void* stream);

/* Network output for n feature rows (device): bf16 = 1 uses the tensor-core
 * path of the collision kernels, bf16 = 0 an FP32 reference on CUDA cores. */
lbm_status lbm_closure_forward(const float* theta, const float* feats, int64_t n, int bf16,
                               float* out, void* stream);

/* Load trained weights (host, n = 5313 FP32) into a multi-resolution grid;
 * with phys.closure = 1 every later step applies the closure on levels >= 1
 * (disaggregated schedule only). */
lbm_status lbm_closure_load(lbm_grid* g, const float* theta, size_t n);

/* ------------------------------------------------------------- batching
 * Not in the paper (a serving-style use of the same update): many
 * independent dense and 8^3 block-sparse grids advance together, one
 * persistent kernel launch per step over a work list of 512-voxel items
 * (dense: consecutive voxel ids; sparse: whole blocks), the steps of one
 * lbm_batch_step call captured once into a CUDA graph and replayed.
 * Cases keep their own state, walls and tau; they must share storage and
 * collision, be D3Q19, have no regularized voxels and fewer than 2^31 / 19
 * voxels (slots) each, dense cases at most 2047 x 2047 x 1023; otherwise
 * lbm_batch_create returns LBM_ERR_UNSUPPORTED.  A
 * case may still be used on its own (lbm_get_moments, lbm_step, ...) between
 * batch steps. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(int n_cases, lbm_grid* const* cases, lbm_batch** out);
lbm_status lbm_batch_destroy(lbm_batch* b);
/* Advance every case by n_steps steps on `stream` (graph replay; the graph
 * for a given n_steps is captured on first use). */
lbm_status lbm_batch_step(lbm_batch* b, int n_steps, void* stream);
/* Autotuner of the persistent grid: times n_steps steps for 1, 2, 3, 4, 6 and
 * 8 CTAs per SM from the current states (restored afterwards), keeps the
 * fastest; *chosen gets it, ms_per_step (6 doubles or NULL) the timings. */
lbm_status lbm_batch_autotune(lbm_batch* b, int n_steps, int* chosen, double* ms_per_step);
/* Learned closure on the small cases of a batch, the same network and
 * parameter layout as lbm_closure_load: every case whose largest edge is at
 * most max_edge collides with tau_eff = max(tau + d_tau, 1/2 + 1e-3) on each
 * fluid voxel, d_tau the network evaluated on the features of the voxel's
 * pulled populations and the case's tau (BF16 weights on tensor cores, FP32
 * accumulation).  theta: host, n = 5313 FP32, copied.  max_edge <= 0 turns
 * the closure off (theta may then be NULL).  Captured graphs are dropped. */
lbm_status lbm_batch_closure_load(lbm_batch* b, const float* theta, size_t n, int max_edge);
lbm_status lbm_batch_info(const lbm_batch* b, int64_t* n_updated, int64_t* n_items,
                          int* ctas_per_sm);

/* Wait for the grid's last stream and return (and clear) the latched device
 * status. */
lbm_status lbm_sync(lbm_grid* g);

/* Per-kernel timing.  lbm_profile(g, 1) clears the records and makes every
 * later kernel launch of this grid record a CUDA event pair on its own
 * stream; lbm_profile(g, 0) stops recording.  lbm_profile_read waits for the
 * grid's stream and aggregates the records per kernel: launches, summed
 * event time and summed units (updated voxels the launches processed).
 * At most `max` entries are written; *n_out receives the number of kernels. */
typedef struct {
  char name[48];
  int64_t launches;
  double total_ms;
  int64_t units;
} lbm_kernel_stat;
lbm_status lbm_profile(lbm_grid* g, int enable);
lbm_status lbm_profile_read(lbm_grid* g, lbm_kernel_stat* out, int max, int* n_out);
/* The same records one by one, in launch order: each launch's kernel name,
 * start and end in ms after the first recorded launch's start (event times
 * on the launch's own stream, so launches on the multi-resolution and
 * boundary-group streams show their overlap) and units.  At most `max`
 * entries are written; *n_out receives the number of launches recorded. */
typedef struct {
  char name[48];
  double start_ms;
  double end_ms;
  int64_t units;
} lbm_kernel_trace;
lbm_status lbm_profile_trace(lbm_grid* g, lbm_kernel_trace* out, int max, int* n_out);

/* Thread-local message of the last error on this thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
