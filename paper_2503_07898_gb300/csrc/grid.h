// grid.h - host-side grid object of liblbm (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// Status helpers -------------------------------------------------------------
void set_error(const std::string& msg);
lbm_status fail(lbm_status s, const std::string& msg);
lbm_status cuda_fail(cudaError_t e, const char* where);
#define LBM_CUDA(call)                                        \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::lbm::cuda_fail(_e, #call); \
  } while (0)

constexpr int kRedCtas = 1216;  // reduction CTAs per level (152 SMs x 8)

// Interior-kernel variants (dense grids): 16-byte vectors, scalar, 8-byte vectors.
enum { VARIANT_VEC16 = 0, VARIANT_SCALAR = 1, VARIANT_VEC8 = 2, VARIANT_VEC4 = 3, N_VARIANTS = 4,
       VARIANT_STAGED = 4 /* block-sparse lean kernel staged by a bulk copy (8^3 blocks) */ };

// Per-level data --------------------------------------------------------------
struct Level {
  // virtual box of this level, in this level's voxel units
  int nx = 0, ny = 0, nz = 0;
  int E = 0;                  // block edge (0 = dense)
  int nbx = 0, nby = 0, nbz = 0;  // virtual block grid
  int64_t n_blocks = 0;       // active blocks (sparse)
  int64_t n_b = 0;            // boundary blocks, stored first (sparse, memory grouping)
  bool bitmask = false;       // sparse: bitmask grouping (all blocks in Morton order)
  int64_t n_slots = 0;        // dense: voxels; sparse: n_blocks * E^3
  int64_t n_updated = 0;      // fluid + regularized voxels
  int64_t n_upd_b = 0;        // updated voxels inside boundary blocks (sparse)
  int64_t n_reg = 0;          // regularized voxels
  size_t pop_bytes = 0;       // bytes of one population buffer (19 arrays)
  void* f[3] = {nullptr, nullptr, nullptr};
  int nbuf = 2;               // 2 (ping-pong) or 3 (ring, multi-resolution levels)
  int cur = 0;                // f[cur] holds the current state
  void* tmp = nullptr;        // multi-resolution unfused schedule: pre-collision buffer

  // multi-resolution
  int64_t n_c = 0;                    // G_c blocks (stored first)
  std::vector<uint8_t> jump_h;        // per block: 0 G_i, 1 finer neighbour, 2 coarser neighbour
  uint8_t* jump_d = nullptr;
  int32_t* coords_d = nullptr;
  std::vector<int32_t> xnbr_coarse_h; // n_blocks x 27
  std::vector<int32_t> xnbr_fine_h;   // n_blocks x 27 x 8
  // interface voxels (a pull leaves the level): slot and the bit set of the
  // directions whose pull does; every other voxel of the level runs the lean
  // kernel, which the per-slot mask keeps off these
  std::vector<int32_t> iface_slot_h;
  std::vector<uint32_t> iface_cross_h;
  int32_t* iface_slot_d = nullptr;
  uint32_t* iface_cross_d = nullptr;
  int64_t n_iface = 0;

  // host tables
  std::vector<uint8_t> flags_h;       // virtual box
  std::vector<int32_t> coords_h;      // n_blocks x 3
  std::vector<int32_t> nbr_h;         // n_blocks x 27
  std::vector<int32_t> bmap_h;        // virtual block grid -> id
  std::vector<float> bc_h;            // 4 per regularized voxel, flag-scan order
  std::vector<uint32_t> bnd_bits_h;   // bitmask grouping: bit b = block b is a boundary block
  std::vector<int32_t> bc_idx_h;      // bitmask grouping: per slot, rank in bc_h or -1

  // device tables
  uint8_t* flags_d = nullptr;    // dense: N (null when all fluid); sparse: n_slots
  uint32_t* wmask_d = nullptr;   // dense, general flags: per-voxel wall mask
  int32_t* reg_list_d = nullptr; // dense: regularized voxel ids (non-contiguous case)
  float4* bc_grp_d = nullptr;    // boundary-group BC values (dense: n_reg; sparse: n_b*E^3)
  float4* bc_full_d = nullptr;   // monolithic kernel: BC for every slot
  int32_t* nbr_d = nullptr;
  int32_t* bmap_d = nullptr;
  uint8_t* blk_walls_d = nullptr; // sparse: 1 if block or its halo has a wall voxel
  uint32_t* bnd_bits_d = nullptr; // bitmask grouping: boundary block bits
  int32_t* reg_blocks_d = nullptr;  // multi-res level 0: blocks holding regularized voxels
  int64_t n_reg_blocks = 0;
  int32_t* bc_idx_d = nullptr;    // bitmask grouping: per-slot index into bc_cmp_d
  float4* bc_cmp_d = nullptr;     // bitmask grouping: BC values, one per regularized voxel

  int variant = VARIANT_SCALAR;   // kernel variant (VARIANT_*), set by lbm_set_variant / autotune

  // dense grouping
  bool dense_has_flags = false;   // any non-fluid voxel
  bool dense_reg_tail = false;    // regularized voxels are exactly the last n_reg ids
};

struct ProfRec {
  int kernel;
  cudaEvent_t a, b;
  int64_t units;
};

struct Grid {
  int kind = 0;  // 0 dense, 1 sparse, 2 multires
  int q = 19;    // lattice: 19 (D3Q19) or 27 (D3Q27)
  lbm_physics phys{};
  lbm_allocator alloc{};
  bool have_alloc = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t stream_ev = nullptr;  // orders a call on a new stream after the previous one
  int n_levels = 1;
  Level lv[4];
  int device = 0;
  int* status_d = nullptr;       // latched device status
  // staged lean kernel: time limit of each CTA's wait for its block copy
  // (lbm_set_wait_limit; past it the CTA latches LBM_ERR_TIMEOUT)
  static constexpr uint64_t kStagedWaitNs = 200000000ull;
  uint64_t staged_wait_ns = kStagedWaitNs;
  double* partials_d = nullptr;  // reduction partials (scratch)
  int n_partials = 0;
  double* sums_d = nullptr;      // 4 doubles
  int64_t steps_done = 0;

  // multi-resolution: a second stream per level for the G_i launch, which
  // overlaps the finer substeps and the G_c launch of its level; the G_c
  // launches (the critical path) run on a high-priority stream
  cudaStream_t mr_aux[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t mr_fork[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t mr_join[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t mr_hi = nullptr;
  cudaEvent_t mr_in = nullptr, mr_out = nullptr;

  // dense / block-sparse grids: the boundary group's kernel runs on its own
  // high-priority stream beside the interior kernel (both read the previous
  // state and write disjoint voxels), forked from and joined back into the
  // step's stream every step
  cudaStream_t grp_hi = nullptr;
  cudaEvent_t grp_fork = nullptr, grp_join = nullptr;

  // learned closure (multi-resolution levels >= 1)
  void* closure_d = nullptr;     // ClosureParams on the device
  bool closure_loaded = false;

  // per-kernel event timing (lbm_profile)
  bool prof = false;
  std::vector<std::string> prof_names;
  std::vector<ProfRec> prof_recs;

  void* dalloc(size_t bytes, cudaStream_t s);
  void dfree(void* p, cudaStream_t s);
};

// Fork the boundary-group stream from s (*hi receives it) / join it back.
lbm_status group_fork(Grid& g, cudaStream_t s, cudaStream_t* hi);
lbm_status group_join(Grid& g, cudaStream_t s);

// Event pair around one kernel launch when profiling is on (else no-op).
int prof_begin(Grid& g, cudaStream_t s, const char* name, int64_t units);
void prof_end(Grid& g, cudaStream_t s, int rec);
void prof_clear(Grid& g);

// Kernel launchers (defined in the .cu files) -------------------------------
// dense.cu, sparse.cu, fields.cu and multires.cu are built once per lattice, into
// namespace q19 (D3Q19) and q27 (D3Q27); the host code picks by Grid::q.
#define LBM_LATTICE_LAUNCHERS                                                              \
  lbm_status dense_step(Grid& g, Level& L, cudaStream_t s);                                \
  /* per-voxel wall mask of a dense level (bits 1..Q-1 wall sources, 30 regularized, */  \
  /* 31 not updated) from L.flags_h */                                                    \
  void dense_wall_mask(const Grid& g, const Level& L, std::vector<uint32_t>& wm);         \
  lbm_status sparse_step(Grid& g, Level& L, cudaStream_t s);                               \
  /* sparse fused kernel over blocks [b0, b1) of L with relaxation omega (no walls) */   \
  lbm_status sparse_uniform_range(Grid& g, Level& L, int64_t b0, int64_t b1, const void* fin, \
                                  void* fout, float omega, cudaStream_t s, const char* name,  \
                                  int64_t units);                                             \
  /* regularized voxels of the blocks listed in L.reg_blocks_d (multi-res level 0) */        \
  lbm_status sparse_reg_blocks(Grid& g, Level& L, const void* fin, void* fout, float omega,   \
                               cudaStream_t s, const char* name);                             \
  lbm_status launch_init_equilibrium(Grid& g, Level& L, const double* rho, const double* u,  \
                                     cudaStream_t s);                                         \
  lbm_status launch_moments(Grid& g, Level& L, double* rho, double* u, cudaStream_t s);     \
  lbm_status launch_decode_f64(Grid& g, Level& L, double* dst, cudaStream_t s);             \
  lbm_status launch_conservation(Grid& g, double* out4, cudaStream_t s);                    \
  lbm_status multires_build(Grid& g, const int finest[3], int n_levels,                      \
                            const uint8_t* level_map);                                       \
  lbm_status multires_finish(Grid& g);                                                       \
  lbm_status multires_step(Grid& g, cudaStream_t s, bool first);                             \
  lbm_status multires_set_boundary(Grid& g, const uint8_t* flags, const float* bc_values,    \
                                   const float* def_bc);
namespace q19 {
LBM_LATTICE_LAUNCHERS
}
namespace q27 {
LBM_LATTICE_LAUNCHERS
}


}  // namespace lbm

struct lbm_grid {
  lbm::Grid g;
};
