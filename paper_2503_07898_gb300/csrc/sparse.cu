// sparse.cu - block-sparse layout (classification + mapping) and the
// per-group fused stream-and-collide kernels.
//
// Disaggregation of a block-sparse grid (Sec. 4, Table 2 "Disag - Mem";
// Sec. 6.2):
//   definition     P_b: the block holds a voxel that needs the regularized
//                  (register-heavy, 3Q) boundary; bounce-back voxels do not
//                  count (Sec. 6.2).
//   classification G_b = boundary blocks, G_nb = the rest.
//   mapping        G_b stored first, then G_nb; inside each group blocks
//                  follow the Morton curve of their coordinates (Sec. 4
//                  orders blocks along a space-filling curve without
//                  naming one).  Storage ((b * Q) + pop) * E^3 + l.
//   operations     sparse_kernel<MODE_INTERIOR> on G_nb (lean, 2Q, bounded
//                  registers); sparse_kernel<MODE_BOUNDARY> on G_b; both
//                  with direct indexing and no per-voxel boundary storage
//                  outside G_b.
// MODE_MONOLITHIC is the paper's naive single kernel: every block, per-voxel
// branches, boundary values read from a full-domain array.
//
// A pull that leaves the block reads the neighbour block through the
// block's row of the 27-entry neighbour table (-1 = no block: bounce-back).  A per-block bit (blk_walls) marks blocks
// that hold or touch a wall voxel or a missing neighbour; only those read
// voxel flags, so uniform fluid blocks stream with no metadata traffic.
#include <algorithm>
#include <numeric>
#include <vector>

#include "d3q19.cuh"
#include "grid.h"
#include "layout.h"
#include "sparse.cuh"

namespace lbm {

#if LBM_Q == 19
// Lattice-independent host code, compiled once (D3Q19 build).
// ------------------------------------------------------------- host layout

static uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

lbm_status sparse_upload(Grid& g, Level& L) {
  auto up = [&](int32_t** dst, const std::vector<int32_t>& src) -> lbm_status {
    *dst = (int32_t*)g.dalloc(src.size() * 4 + 4, g.stream);
    if (!*dst) return fail(LBM_ERR_OOM, "device allocation failed");
    if (!src.empty()) LBM_CUDA(cudaMemcpy(*dst, src.data(), src.size() * 4, cudaMemcpyHostToDevice));
    return LBM_OK;
  };
  lbm_status st;
  if ((st = up(&L.nbr_d, L.nbr_h)) || (st = up(&L.bmap_d, L.bmap_h))) return st;
  return LBM_OK;
}

// Regularized voxels in flag-scan order -> (slot, k).
template <class F> static void for_each_reg(const Level& L, F&& fn) {
  const int E = L.E;
  const int64_t E3 = (int64_t)E * E * E;
  int64_t k = 0;
  for (int z = 0; z < L.nz; ++z)
    for (int y = 0; y < L.ny; ++y)
      for (int x = 0; x < L.nx; ++x) {
        const uint8_t f = L.flags_h[x + (size_t)L.nx * (y + (size_t)L.ny * z)];
        if (!type_regularized(flag_type(f))) continue;
        const int b = L.bmap_h[x / E + (size_t)L.nbx * (y / E + (size_t)L.nby * (z / E))];
        const int64_t slot = (int64_t)b * E3 + (x % E) + E * ((y % E) + E * (z % E));
        fn(slot, k++);
      }
}

lbm_status sparse_set_bc(Grid& g, Level& L, const float* bc_values, const float* def_bc) {
  if (L.n_reg > 0 && !bc_values && !def_bc)
    return fail(LBM_ERR_INVALID, "regularized voxels need bc_values or default_bc");
  const int64_t E3 = (int64_t)L.E * L.E * L.E;
  L.bc_h.assign((size_t)L.n_reg * 4, 0.f);
  if (L.bitmask || g.kind == 2) {
    // indirect indexing: a per-slot rank into one compact value per
    // regularized voxel (flag-scan order)
    L.bc_idx_h.assign((size_t)L.n_slots, -1);
    std::vector<float4> cmp((size_t)L.n_reg);
    for_each_reg(L, [&](int64_t slot, int64_t k) {
      const float* v = bc_values ? bc_values + k * 4 : def_bc;
      for (int c = 0; c < 4; ++c) L.bc_h[(size_t)k * 4 + c] = v[c];
      cmp[(size_t)k] = make_float4(v[0], v[1], v[2], v[3]);
      L.bc_idx_h[(size_t)slot] = (int32_t)k;
    });
    g.dfree(L.bc_idx_d, g.stream);
    g.dfree(L.bc_cmp_d, g.stream);
    g.dfree(L.bc_full_d, g.stream);
    L.bc_full_d = nullptr;
    L.bc_idx_d = (int32_t*)g.dalloc(L.bc_idx_h.size() * 4 + 4, g.stream);
    L.bc_cmp_d = (float4*)g.dalloc(cmp.size() * sizeof(float4) + 16, g.stream);
    if (!L.bc_idx_d || !L.bc_cmp_d) return fail(LBM_ERR_OOM, "device allocation failed");
    if (!L.bc_idx_h.empty())
      LBM_CUDA(cudaMemcpy(L.bc_idx_d, L.bc_idx_h.data(), L.bc_idx_h.size() * 4, cudaMemcpyHostToDevice));
    if (!cmp.empty())
      LBM_CUDA(cudaMemcpy(L.bc_cmp_d, cmp.data(), cmp.size() * sizeof(float4), cudaMemcpyHostToDevice));
    return LBM_OK;
  }
  std::vector<float4> grp((size_t)(L.n_b * E3), make_float4(0.f, 0.f, 0.f, 1.f));
  for_each_reg(L, [&](int64_t slot, int64_t k) {
    const float* v = bc_values ? bc_values + k * 4 : def_bc;
    for (int c = 0; c < 4; ++c) L.bc_h[(size_t)k * 4 + c] = v[c];
    grp[(size_t)slot] = make_float4(v[0], v[1], v[2], v[3]);
  });
  g.dfree(L.bc_grp_d, g.stream);
  g.dfree(L.bc_full_d, g.stream);
  L.bc_full_d = nullptr;
  L.bc_grp_d = (float4*)g.dalloc(grp.size() * sizeof(float4) + 16, g.stream);
  if (!L.bc_grp_d) return fail(LBM_ERR_OOM, "device allocation failed");
  if (!grp.empty())
    LBM_CUDA(cudaMemcpy(L.bc_grp_d, grp.data(), grp.size() * sizeof(float4), cudaMemcpyHostToDevice));
  return LBM_OK;
}

void sparse_fill_bc_full(const Level& L, float4* full) {
  for_each_reg(L, [&](int64_t slot, int64_t k) {
    full[slot] = make_float4(L.bc_h[k * 4], L.bc_h[k * 4 + 1], L.bc_h[k * 4 + 2], L.bc_h[k * 4 + 3]);
  });
}

#endif  // LBM_Q == 19

namespace LBM_LNS {

lbm_status sparse_build(Grid& g, Level& L) {
  const int E = L.E;
  L.nbx = (L.nx + E - 1) / E;
  L.nby = (L.ny + E - 1) / E;
  L.nbz = (L.nz + E - 1) / E;
  if (L.nbx > 1024 || L.nby > 1024 || L.nbz > 1024)
    return fail(LBM_ERR_INVALID, "more than 1024 blocks along an axis");
  const int64_t nvb = (int64_t)L.nbx * L.nby * L.nbz;
  std::vector<uint8_t> act((size_t)nvb, 0), bnd((size_t)nvb, 0), wallb((size_t)nvb, 0);
  int64_t n_upd = 0, n_reg = 0, n_upd_b = 0;
  for (int z = 0; z < L.nz; ++z)
    for (int y = 0; y < L.ny; ++y)
      for (int x = 0; x < L.nx; ++x) {
        const uint8_t f = L.flags_h[x + (size_t)L.nx * (y + (size_t)L.ny * z)];
        const int t = flag_type(f);
        if (!type_updated(t) && !type_wall(t)) return fail(LBM_ERR_INVALID, "unknown voxel type");
        if (type_regularized(t) && flag_normal(f) > 5)
          return fail(LBM_ERR_INVALID, "regularized voxel with bad normal");
        const int64_t vb = x / E + (int64_t)L.nbx * (y / E + (int64_t)L.nby * (z / E));
        if (type_updated(t)) act[(size_t)vb] = 1;
        if (type_regularized(t)) bnd[(size_t)vb] = 1;
        if (type_wall(t)) wallb[(size_t)vb] = 1;
      }
  // voxels of a partial block beyond the box edge are "not in domain"
  if (L.nx % E || L.ny % E || L.nz % E)
    for (int64_t vb = 0; vb < nvb; ++vb) {
      const int bx = (int)(vb % L.nbx), by = (int)((vb / L.nbx) % L.nby), bz = (int)(vb / ((int64_t)L.nbx * L.nby));
      if ((bx + 1) * E > L.nx || (by + 1) * E > L.ny || (bz + 1) * E > L.nz) wallb[(size_t)vb] = 1;
    }
  std::vector<int64_t> ids;
  for (int64_t vb = 0; vb < nvb; ++vb)
    if (act[(size_t)vb]) ids.push_back(vb);
  // memory grouping: boundary blocks first; bitmask grouping: Morton only
  L.bitmask = g.phys.schedule == LBM_SCHEDULE_BITMASK;
  auto key = [&](int64_t vb) {
    const uint32_t bx = (uint32_t)(vb % L.nbx), by = (uint32_t)((vb / L.nbx) % L.nby),
                   bz = (uint32_t)(vb / ((int64_t)L.nbx * L.nby));
    const uint64_t grp = L.bitmask ? 0 : (bnd[(size_t)vb] ? 0 : 1);
    return (grp << 32) | morton3(bx, by, bz);
  };
  std::sort(ids.begin(), ids.end(), [&](int64_t a, int64_t b) { return key(a) < key(b); });
  L.n_blocks = (int64_t)ids.size();
  L.n_b = 0;
  for (int64_t vb : ids) L.n_b += bnd[(size_t)vb] ? 1 : 0;
  auto is_bnd = [&](int64_t b) { return bnd[(size_t)ids[(size_t)b]] != 0; };
  L.bnd_bits_h.assign(L.bitmask ? (size_t)((L.n_blocks + 31) / 32) : 0, 0u);
  if (L.bitmask)
    for (int64_t b = 0; b < L.n_blocks; ++b)
      if (is_bnd(b)) L.bnd_bits_h[(size_t)(b / 32)] |= 1u << (b % 32);
  L.bmap_h.assign((size_t)nvb, -1);
  L.coords_h.resize((size_t)L.n_blocks * 3);
  for (int64_t b = 0; b < L.n_blocks; ++b) {
    const int64_t vb = ids[(size_t)b];
    L.bmap_h[(size_t)vb] = (int32_t)b;
    L.coords_h[(size_t)b * 3 + 0] = (int32_t)(vb % L.nbx);
    L.coords_h[(size_t)b * 3 + 1] = (int32_t)((vb / L.nbx) % L.nby);
    L.coords_h[(size_t)b * 3 + 2] = (int32_t)(vb / ((int64_t)L.nbx * L.nby));
  }
  const int* per = g.phys.periodic;
  const int nbd[3] = {L.nbx, L.nby, L.nbz};
  L.nbr_h.assign((size_t)L.n_blocks * 27, -1);
  for (int64_t b = 0; b < L.n_blocks; ++b) {
    for (int k = 0; k < 27; ++k) {
      int q[3] = {L.coords_h[b * 3] + k % 3 - 1, L.coords_h[b * 3 + 1] + (k / 3) % 3 - 1,
                  L.coords_h[b * 3 + 2] + k / 9 - 1};
      bool ok = true;
      for (int a = 0; a < 3; ++a)
        if (q[a] < 0 || q[a] >= nbd[a]) {
          if (per[a]) q[a] = (q[a] + nbd[a]) % nbd[a];
          else ok = false;
        }
      if (ok) L.nbr_h[(size_t)b * 27 + k] = L.bmap_h[q[0] + (size_t)L.nbx * (q[1] + (size_t)L.nby * q[2])];
    }
  }
  // a block needs flag reads when it, or any of its 26 neighbours, holds a
  // wall voxel, or when a neighbour block is missing
  const int64_t E3 = (int64_t)E * E * E;
  std::vector<uint8_t> bw((size_t)L.n_blocks, 0);
  for (int64_t b = 0; b < L.n_blocks; ++b) {
    bool w = wallb[(size_t)ids[(size_t)b]] != 0;
    for (int k = 0; k < 27 && !w; ++k) {
      const int32_t nb = L.nbr_h[(size_t)b * 27 + k];
      if (nb < 0 || wallb[(size_t)ids[(size_t)nb]]) w = true;
    }
    bw[(size_t)b] = w ? 1 : 0;
  }
  L.n_slots = L.n_blocks * E3;
  std::vector<uint8_t> sf((size_t)L.n_slots, (uint8_t)T_OUTSIDE);
  for (int64_t b = 0; b < L.n_blocks; ++b) {
    const int bx = L.coords_h[b * 3], by = L.coords_h[b * 3 + 1], bz = L.coords_h[b * 3 + 2];
    for (int l = 0; l < E3; ++l) {
      const int x = bx * E + l % E, y = by * E + (l / E) % E, z = bz * E + l / (E * E);
      if (x < L.nx && y < L.ny && z < L.nz) {
        const uint8_t f = L.flags_h[x + (size_t)L.nx * (y + (size_t)L.ny * z)];
        sf[(size_t)(b * E3 + l)] = f;
        if (type_updated(flag_type(f))) {
          ++n_upd;
          if (is_bnd(b)) ++n_upd_b;
        }
        if (type_regularized(flag_type(f))) ++n_reg;
      }
    }
  }
  L.n_updated = n_upd;
  L.n_upd_b = n_upd_b;
  L.n_reg = n_reg;
  // per-slot wall mask of the blocks that pull with checks (walls bit or
  // boundary group): bit i = the source of population i bounces back (missing
  // block or wall voxel), bit 30 = regularized voxel, bit 31 = not updated.
  // One coalesced 32-bit load then replaces a flag load per population.
  std::vector<uint32_t> wm((size_t)L.n_slots, 0u);
  for (int64_t b = 0; b < L.n_blocks; ++b) {
    if (!bw[(size_t)b] && !is_bnd(b)) continue;
    for (int l = 0; l < E3; ++l) {
      const int t = flag_type(sf[(size_t)(b * E3 + l)]);
      uint32_t m = 0;
      if (!type_updated(t)) m |= 1u << 31;
      if (type_regularized(t)) m |= 1u << 30;
      const int lc[3] = {l % E, (l / E) % E, l / (E * E)};
      for (int i = 1; i < Q; ++i) {
        int sc[3] = {lc[0] - cx(i), lc[1] - cy(i), lc[2] - cz(i)};
        int d[3];
        for (int a = 0; a < 3; ++a) {
          d[a] = sc[a] < 0 ? -1 : (sc[a] >= E ? 1 : 0);
          sc[a] -= d[a] * E;
        }
        const int32_t nb = L.nbr_h[(size_t)b * 27 + (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1)];
        const bool wall =
            nb < 0 || type_wall(flag_type(sf[(size_t)((int64_t)nb * E3 + sc[0] + E * (sc[1] + E * sc[2]))]));
        if (wall) m |= 1u << i;
      }
      wm[(size_t)(b * E3 + l)] = m;
    }
  }
  // stash the per-slot flags, masks and wall bits until upload
  L.bc_h.clear();
  g.dfree(L.flags_d, g.stream);
  g.dfree(L.blk_walls_d, g.stream);
  g.dfree(L.wmask_d, g.stream);
  L.flags_d = (uint8_t*)g.dalloc(sf.size(), g.stream);
  L.blk_walls_d = (uint8_t*)g.dalloc(bw.size() ? bw.size() : 1, g.stream);
  L.wmask_d = (uint32_t*)g.dalloc(wm.size() * 4 + 4, g.stream);
  if (!L.flags_d || !L.blk_walls_d || !L.wmask_d) return fail(LBM_ERR_OOM, "device allocation failed");
  LBM_CUDA(cudaMemcpy(L.flags_d, sf.data(), sf.size(), cudaMemcpyHostToDevice));
  if (!bw.empty()) LBM_CUDA(cudaMemcpy(L.blk_walls_d, bw.data(), bw.size(), cudaMemcpyHostToDevice));
  if (!wm.empty()) LBM_CUDA(cudaMemcpy(L.wmask_d, wm.data(), wm.size() * 4, cudaMemcpyHostToDevice));
  if (L.bitmask) {
    g.dfree(L.bnd_bits_d, g.stream);
    L.bnd_bits_d = (uint32_t*)g.dalloc(L.bnd_bits_h.size() * 4 + 4, g.stream);
    if (!L.bnd_bits_d) return fail(LBM_ERR_OOM, "device allocation failed");
    if (!L.bnd_bits_h.empty())
      LBM_CUDA(cudaMemcpy(L.bnd_bits_d, L.bnd_bits_h.data(), L.bnd_bits_h.size() * 4,
                          cudaMemcpyHostToDevice));
  }
  return LBM_OK;
}

// ------------------------------------------------------------------ kernels

// INTERIOR / BOUNDARY: the two group kernels of the memory grouping, each
// over its own contiguous block range; *_BM: the same kernels under the
// bitmask grouping, launched over every block and returning at once on a
// block of the other group; MONOLITHIC: the naive single kernel.
// REG_LIST: the regularized voxels (only) of a list of 8^3 blocks whose other
// voxels an INTERIOR launch updates (multi-resolution level 0 with a lid).
enum { MODE_INTERIOR = 0, MODE_BOUNDARY = 1, MODE_MONOLITHIC = 2, MODE_INTERIOR_BM = 3,
       MODE_BOUNDARY_BM = 4, MODE_REG_LIST = 5 };
constexpr int SP_THREADS = 256;

struct SparseArgs {
  const void* fin;
  void* fout;
  const int32_t* nbr;
  const uint8_t* flags;
  const uint32_t* wmask;  // per-slot wall mask (blocks with walls, boundary group)
  const uint8_t* blk_walls;
  const float4* bc;
  const int32_t* blist;      // REG_LIST: block ids (two CTAs per block)
  const uint32_t* bnd_bits;  // bitmask grouping: boundary block bits
  const int32_t* bc_idx;     // bitmask grouping: per-slot index into bc_cmp
  const float4* bc_cmp;      // bitmask grouping: compact BC values
  int64_t s0, s1;  // slot range [s0, s1), block aligned
  float omega;
  int* status;     // latched device status (staged kernel: a bulk copy that never lands)
  uint64_t wait_ns;  // staged kernel: limit of the wait for the block copy
};

// ---------------------------------------------- bulk-copy staging (TMA)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive once and announce `bytes` of asynchronous copy completing the phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16), completion counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait on phase `parity`, bounded by time: false once limit_ns have passed
// without the phase completing (limit_ns = 0: false at once, no poll).
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return false;
  const uint64_t t0 = global_ns();
  do {
    if (mbar_try_wait(bar, parity)) return true;
  } while (global_ns() - t0 < limit_ns);
  return false;
}
// After a wait has given up, the CTA must not exit while its bulk copy may
// still write its shared memory: it drains the copy for up to this long.  A
// 19 KB (D3Q27 FP32: 55 KB) block copy lands within microseconds, so one
// second covers any copy that is in flight; only a copy that never
// completes (a lost transfer) can outlast it, and then the CTA leaves
// rather than hang the device.
constexpr uint64_t STAGED_DRAIN_NS = 1000000000ull;

// One voxel (slot) of the group the mode selects.
template <int S, int E, int COLL, int MODE, class IDX = int64_t>
__device__ __forceinline__ void sparse_update(const SparseArgs& a, int64_t slot) {
  using T = typename Codec<S>::T;
  constexpr int E3 = E * E * E;
  constexpr bool LEAN = MODE == MODE_INTERIOR || MODE == MODE_INTERIOR_BM;
  const int64_t b = slot / E3;
  const int l = (int)(slot - b * E3);
  if constexpr (MODE == MODE_INTERIOR_BM || MODE == MODE_BOUNDARY_BM) {
    const bool bnd = (a.bnd_bits[b >> 5] >> (b & 31)) & 1u;
    if (bnd != (MODE == MODE_BOUNDARY_BM)) return;
  }
  const bool walls = !LEAN || a.blk_walls[b];
  uint32_t wm = 0;
  if (walls) {
    wm = a.wmask[slot];
    // lean kernels leave regularized voxels to a boundary launch
    if (wm & (LEAN ? 0xC0000000u : 0x80000000u)) return;
    if (MODE == MODE_REG_LIST && !(wm & (1u << 30))) return;
  }
  const T* __restrict__ fin = (const T*)a.fin;
  float g[Q];
  sparse_pull_voxel<S, E, IDX>(fin, a.nbr + b * 27, wm, b, l, walls, g);
  if constexpr (LEAN) {
    collide<COLL>(g, a.omega);
  } else {
    if (wm & (1u << 30)) {
      const uint8_t own = a.flags[slot];
      const float4 bc = (MODE == MODE_BOUNDARY_BM || MODE == MODE_REG_LIST)
                            ? a.bc_cmp[a.bc_idx[slot]] : a.bc[slot];
      regularized_node(g, flag_type(own), flag_normal(own), bc, a.omega);
    } else {
      collide<COLL>(g, a.omega);
    }
  }
  T* __restrict__ fout = (T*)a.fout;
  const IDX o = (IDX)b * (IDX)(Q * E3) + (IDX)l;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    fout[o + (IDX)(I * E3)] = Codec<S>::template store<I>(g[I]);
  });
}

// BOUNDARY_BM with 8^3 blocks takes one block per CTA (two voxels per
// thread): the launch over every block, most of which leave at once on
// their boundary bit, then has half as many CTAs.
// Resident CTAs per SM of the lean kernels: the 16-bit, 32-bit-offset D3Q19
// form fits in 40 registers without spilling and runs 6 (measured +6 % on
// the FP16 sphere channel against 5); with 64-bit offsets it stays at 5.
template <int S, int MODE, class IDX>
constexpr int sparse_min_ctas() {
  return (MODE == MODE_INTERIOR || MODE == MODE_INTERIOR_BM)
             ? (Q == 27 ? 3 : (S == S_F32 ? 4 : (MODE == MODE_INTERIOR && sizeof(IDX) == 4 ? 6 : 5)))
             : 1;
}

template <int S, int E, int COLL, int MODE, class IDX = int64_t>
__global__ void __launch_bounds__(SP_THREADS, sparse_min_ctas<S, MODE, IDX>())
    sparse_kernel(SparseArgs a) {
  constexpr int E3 = E * E * E;
  if constexpr (MODE == MODE_BOUNDARY_BM && E3 == 2 * SP_THREADS) {
    const int64_t b = blockIdx.x;
    if (!((a.bnd_bits[b >> 5] >> (b & 31)) & 1u)) return;  // uniform per CTA
    sparse_update<S, E, COLL, MODE, IDX>(a, b * E3 + threadIdx.x);
    sparse_update<S, E, COLL, MODE, IDX>(a, b * E3 + SP_THREADS + threadIdx.x);
  } else {
    int64_t slot;
    if constexpr (MODE == MODE_REG_LIST)
      slot = (int64_t)a.blist[blockIdx.x >> 1] * E3 + (blockIdx.x & 1) * SP_THREADS + threadIdx.x;
    else
      slot = a.s0 + (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    if (slot >= a.s1) return;
    sparse_update<S, E, COLL, MODE, IDX>(a, slot);
  }
}

// Two-voxel form of the lean interior kernel for 16-bit storage (D3Q19, 8^3
// blocks, 32-bit offsets).  A CTA updates one block; thread t takes the two
// voxels 2t and 2t + 1, neighbours along x (lx = 2k, 2k + 1, k = t mod 4),
// so a warp holds one z plane of the block:
//  - the pulls with c_x = 0 of the two voxels are adjacent and aligned (the
//    element offset of each term is even): one 32-bit load brings both;
//  - of the pulls with c_x = +1 only the first voxel's can cross the -x face
//    (k = 0), of those with c_x = -1 only the second voxel's the +x face
//    (k = 3); the other voxel's source is in the block it would reach
//    without the x move;
//  - the 27 neighbour offsets are read once per CTA into shared memory, and
//    the block choices by (c_y, c_z) are formed once per thread and shared
//    by both voxels;
//  - the results go out as one 32-bit store of both voxels per population
//    (cvt.rn.{f16,bf16}x2.f32 packs them).
// Blocks with a wall bit (a wall voxel in or next to the block, a missing
// neighbour, masked voxels) read the wall masks of their voxels, and the
// choice is made per warp, which holds one z plane of 64 voxels in either
// form: a warp in which no voxel has a bit runs the two-voxel form, any
// other warp the one-voxel update of the plane's voxels 64w + lane and
// 64w + 32 + lane.  (Measured on GB300, FP16: the one-voxel update for
// every warp of such blocks gave sphere channel 53.3, 384^3 cavity 59.3,
// turbulence 55.1 GLUPS; a two-voxel wall form for the warps with bits
// (bounce-back source selects, a warp vote per c_x = 0 pair load, unpaired
// stores next to masked voxels) 51.6, 56.3, 57.8; running the wall blocks
// as a second launch of the one-voxel kernel over a block list was 3-4 %
// slower on every 16-bit workload.)
template <int S> struct Pair16;
template <> struct Pair16<S_F16> {
  using T2 = __half2;
  __device__ static __forceinline__ float lo(T2 v) { return __low2float(v); }
  __device__ static __forceinline__ float hi(T2 v) { return __high2float(v); }
  __device__ static __forceinline__ T2 pack(float a, float b) { return __floats2half2_rn(a, b); }
};
template <> struct Pair16<S_BF16> {
  using T2 = __nv_bfloat162;
  __device__ static __forceinline__ float lo(T2 v) { return __low2float(v); }
  __device__ static __forceinline__ float hi(T2 v) { return __high2float(v); }
  __device__ static __forceinline__ T2 pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

template <int S, int COLL>
__global__ void __launch_bounds__(SP_THREADS, 4) sparse_pair16(SparseArgs a) {
  static_assert(Q == 19 && S != S_F32, "two-voxel kernel: D3Q19, 16-bit storage");
  using T = typename Codec<S>::T;
  using P = Pair16<S>;
  using T2 = typename P::T2;
  constexpr int E3 = 512, QE3 = Q * E3;
  __shared__ int32_t nb_off[27];
  const int b = (int)(a.s0 / E3) + (int)blockIdx.x;
  const int t = threadIdx.x;
  if (t < 27) nb_off[t] = __ldg(a.nbr + (int64_t)b * 27 + t) * QE3;
  __syncthreads();
  if (a.blk_walls[b]) {  // uniform per CTA
    const uint32_t* wm = a.wmask + (int64_t)b * E3 + 2 * t;
    if (__any_sync(0xffffffffu, (wm[0] | wm[1]) != 0u)) {  // uniform per warp
      const int64_t s = (int64_t)b * E3 + 2 * (t & ~31) + (t & 31);
      sparse_update<S, 8, COLL, MODE_INTERIOR, int32_t>(a, s);
      sparse_update<S, 8, COLL, MODE_INTERIOR, int32_t>(a, s + 32);
      return;
    }
  }
  const int k = t & 3, ly = (t >> 2) & 7, lz = t >> 5;
  const int ey = ly == 0 ? -1 : (ly == 7 ? 1 : 0);
  const int ez = lz == 0 ? -1 : (lz == 7 ? 1 : 0);
  const bool xa = k == 0, xb = k == 3;  // first voxel at lx = 0, second at lx = 7
  const int oS = b * QE3;
  const int oY = nb_off[13 + 3 * ey], oZ = nb_off[13 + 9 * ez], oYZ = nb_off[13 + 3 * ey + 9 * ez];
  // across the -x face (first voxel) and the +x face (second voxel)
  const int oXm = nb_off[12], oXYm = nb_off[12 + 3 * ey], oXZm = nb_off[12 + 9 * ez];
  const int oXp = nb_off[14], oXYp = nb_off[14 + 3 * ey], oXZp = nb_off[14 + 9 * ez];
  // in-block source coordinate parts for c = +1, 0, -1 (pre-scaled)
  const int yp = ((ly - 1) & 7) * 8, y0 = ly * 8, yn = ((ly + 1) & 7) * 8;
  const int zp = ((lz - 1) & 7) * 64, z0 = lz * 64, zn = ((lz + 1) & 7) * 64;
  const int lxa = 2 * k;
  const T* __restrict__ fin = (const T*)a.fin;
  float ga[Q], gb[Q];
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    const bool ky = Y != 0 && ey == -Y, kz = Z != 0 && ez == -Z;
    // block reached by the (c_y, c_z) move alone
    const int oyz = (Y != 0 && Z != 0) ? (ky ? (kz ? oYZ : oY) : (kz ? oZ : oS))
                                       : (Y != 0 ? (ky ? oY : oS) : (Z != 0 ? (kz ? oZ : oS) : oS));
    const int lyz = (Y > 0 ? yp : (Y < 0 ? yn : y0)) + (Z > 0 ? zp : (Z < 0 ? zn : z0));
    if constexpr (X == 0) {
      const T2 w = reinterpret_cast<const T2*>(fin)[(oyz + I * E3 + lyz + lxa) >> 1];
      ga[I] = P::lo(w);
      gb[I] = P::hi(w);
    } else if constexpr (X > 0) {
      // first voxel: source lx - 1 (7 of the -x block when k = 0); second: lx - 1 = 2k
      const int ox = Y != 0 ? (ky ? oXYm : oXm) : (Z != 0 ? (kz ? oXZm : oXm) : oXm);
      const int oa = xa ? ox : oyz;
      ga[I] = Codec<S>::template load<I>(fin[oa + I * E3 + lyz + ((lxa - 1) & 7)]);
      gb[I] = Codec<S>::template load<I>(fin[oyz + I * E3 + lyz + lxa]);
    } else {
      // first voxel: source lx + 1 = 2k + 1; second: 2k + 2 (0 of the +x block when k = 3)
      const int ox = Y != 0 ? (ky ? oXYp : oXp) : (Z != 0 ? (kz ? oXZp : oXp) : oXp);
      const int ob = xb ? ox : oyz;
      ga[I] = Codec<S>::template load<I>(fin[oyz + I * E3 + lyz + lxa + 1]);
      gb[I] = Codec<S>::template load<I>(fin[ob + I * E3 + lyz + ((lxa + 2) & 7)]);
    }
  });
  collide<COLL>(ga, a.omega);
  collide<COLL>(gb, a.omega);
  T2* __restrict__ out = reinterpret_cast<T2*>(a.fout) + (oS >> 1) + t;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    out[I * (E3 / 2)] = P::pack(ga[I], gb[I]);
  });
}

// Pull of voxel l of block b with the block's populations staged in shared
// memory (sb): in-block sources come from there, sources across the block's
// faces from global memory; block selection and wall rule as in
// sparse_pull_voxel_t (8^3 blocks).
template <int S, bool WALLS>
__device__ __forceinline__ void staged_pull(const typename Codec<S>::T* sb,
                                            const typename Codec<S>::T* __restrict__ fin,
                                            const int32_t* nbr27, uint32_t wm, int b, int l,
                                            float g[Q]) {
  using T = typename Codec<S>::T;
  constexpr int E = 8, E3 = 512, M = 7;
  const int lx = l & M, ly = (l / E) & M, lz = l / (E * E);
  const int ex = lx == 0 ? -1 : (lx == M ? 1 : 0);
  const int ey = ly == 0 ? -1 : (ly == M ? 1 : 0);
  const int ez = lz == 0 ? -1 : (lz == M ? 1 : 0);
  const int nX = __ldg(nbr27 + 13 + ex), nY = __ldg(nbr27 + 13 + 3 * ey);
  const int nZ = __ldg(nbr27 + 13 + 9 * ez);
  const int nXY = __ldg(nbr27 + 13 + ex + 3 * ey), nXZ = __ldg(nbr27 + 13 + ex + 9 * ez);
  const int nYZ = __ldg(nbr27 + 13 + 3 * ey + 9 * ez);
  const int nXYZ = Q == 27 ? __ldg(nbr27 + 13 + ex + 3 * ey + 9 * ez) : b;
  const int xp = (lx - 1) & M, xn = (lx + 1) & M;
  const int yp = ((ly - 1) & M) * E, yn = ((ly + 1) & M) * E, y0 = ly * E;
  const int zp = ((lz - 1) & M) * E * E, zn = ((lz + 1) & M) * E * E, z0 = lz * E * E;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    const bool kx = X != 0 && ex == -X;
    const bool ky = Y != 0 && ey == -Y;
    const bool kz = Z != 0 && ez == -Z;
    int nb = b;
    if constexpr (X != 0 && Y != 0 && Z != 0)
      nb = kz ? (kx ? (ky ? nXYZ : nXZ) : (ky ? nYZ : nZ)) : (kx ? (ky ? nXY : nX) : (ky ? nY : b));
    else if constexpr (X != 0 && Y != 0) nb = kx ? (ky ? nXY : nX) : (ky ? nY : b);
    else if constexpr (X != 0 && Z != 0) nb = kx ? (kz ? nXZ : nX) : (kz ? nZ : b);
    else if constexpr (Y != 0 && Z != 0) nb = ky ? (kz ? nYZ : nY) : (kz ? nZ : b);
    else if constexpr (X != 0) nb = kx ? nX : b;
    else if constexpr (Y != 0) nb = ky ? nY : b;
    else if constexpr (Z != 0) nb = kz ? nZ : b;
    const int ls = (X > 0 ? xp : (X < 0 ? xn : lx)) + (Y > 0 ? yp : (Y < 0 ? yn : y0)) +
                   (Z > 0 ? zp : (Z < 0 ? zn : z0));
    const bool out = kx || ky || kz;
    T v;
    if (WALLS && ((wm >> I) & 1u)) v = sb[opp(I) * E3 + l];
    else if (out) v = fin[(int64_t)nb * (Q * E3) + (I * E3 + ls)];
    else v = sb[I * E3 + ls];
    g[I] = Codec<S>::template load<I>(v);
  });
}

// Lean (interior-group) step with each 8^3 block staged in shared memory by
// one bulk asynchronous copy: thread 0 arms the CTA's mbarrier with the
// block's byte count and issues the copy, every thread waits on the barrier
// (bounded), then updates two voxels (z-halves of the block).
template <int S, int COLL>
__global__ void __launch_bounds__(SP_THREADS, Q == 27 ? 3 : (S == S_F32 ? 4 : 5))
    sparse_staged(SparseArgs a) {
  using T = typename Codec<S>::T;
  constexpr int E3 = 512;
  constexpr uint32_t BYTES = (uint32_t)(Q * E3 * sizeof(T));
  extern __shared__ __align__(128) unsigned char st_smem[];
  __shared__ __align__(8) uint64_t bar;
  T* sb = reinterpret_cast<T*>(st_smem);
  const int64_t b = a.s0 / E3 + blockIdx.x;
  const T* __restrict__ fin = (const T*)a.fin;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_arrive_expect_tx(&bar, BYTES);
    bulk_g2s(sb, fin + b * (Q * E3), BYTES, &bar);
  }
  __syncthreads();
  if (!mbar_wait_ns(&bar, 0, a.wait_ns)) {
    // the block is not updated this step: latch the timeout, then drain the
    // copy (it may still be in flight into this CTA's shared memory) before
    // the CTA gives that memory up
    if (a.status) atomicExch(a.status, (int)LBM_ERR_TIMEOUT);
    mbar_wait_ns(&bar, 0, STAGED_DRAIN_NS);
    return;
  }
  const bool walls = a.blk_walls[b] != 0;
  T* __restrict__ fout = (T*)a.fout;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int l = h * SP_THREADS + threadIdx.x;
    uint32_t wm = 0;
    if (walls) {
      wm = a.wmask[b * E3 + l];
      if (wm & 0xC0000000u) continue;  // not updated, or a regularized voxel of another launch
    }
    float g[Q];
    if (walls) staged_pull<S, true>(sb, fin, a.nbr + b * 27, wm, (int)b, l, g);
    else staged_pull<S, false>(sb, fin, a.nbr + b * 27, 0u, (int)b, l, g);
    collide<COLL>(g, a.omega);
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      fout[(b * Q + I) * E3 + l] = Codec<S>::template store<I>(g[I]);
    });
  }
}

template <int S, int COLL>
static void launch_staged(Grid& g, SparseArgs a, cudaStream_t s, const char* name, int64_t units) {
  if (a.s1 <= a.s0) return;
  using T = typename Codec<S>::T;
  constexpr int BYTES = (int)(Q * 512 * sizeof(T));
  static bool opted_in = false;  // more than 48 KB of dynamic shared memory with D3Q27 FP32
  if (!opted_in) {
    cudaFuncSetAttribute(sparse_staged<S, COLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES);
    opted_in = true;
  }
  a.status = g.status_d;
  a.wait_ns = g.staged_wait_ns;
  const int pr = prof_begin(g, s, name, units);
  sparse_staged<S, COLL><<<(unsigned)((a.s1 - a.s0) / 512), SP_THREADS, BYTES, s>>>(a);
  prof_end(g, s, pr);
}

template <int S, int COLL>
static void reg_list_t(Grid& g, Level& L, const void* fin, void* fout, float omega, cudaStream_t s,
                       const char* name) {
  SparseArgs a{};
  a.fin = fin;
  a.fout = fout;
  a.nbr = L.nbr_d;
  a.flags = L.flags_d;
  a.wmask = L.wmask_d;
  a.blk_walls = L.blk_walls_d;
  a.blist = L.reg_blocks_d;
  a.bc_idx = L.bc_idx_d;
  a.bc_cmp = L.bc_cmp_d;
  a.omega = omega;
  a.s0 = 0;
  a.s1 = L.n_blocks * 512;
  const int pr = prof_begin(g, s, name, L.n_reg);
  sparse_kernel<S, 8, COLL, MODE_REG_LIST><<<(unsigned)(2 * L.n_reg_blocks), SP_THREADS, 0, s>>>(a);
  prof_end(g, s, pr);
}

// i32: the level's Q E^3 n_blocks population elements fit in 31 bits, so the
// lean kernel indexes with 32-bit offsets (fewer integer instructions per
// pull); the other modes keep 64-bit indexing.
template <int S, int E, int COLL, int MODE>
static void launch_range(Grid& g, SparseArgs a, cudaStream_t s, const char* name, int64_t units,
                         bool i32 = false) {
  if (a.s1 <= a.s0) return;
  constexpr int64_t E3 = (int64_t)E * E * E;
  const unsigned nb = (MODE == MODE_BOUNDARY_BM && E3 == 2 * SP_THREADS)
                          ? (unsigned)((a.s1 - a.s0) / E3)  // one CTA per block
                          : (unsigned)((a.s1 - a.s0 + SP_THREADS - 1) / SP_THREADS);
  const int pr = prof_begin(g, s, name, units);
  bool pair = false;
  if constexpr (MODE == MODE_INTERIOR && E == 8 && S != S_F32 && Q == 19) {
    // 16-bit storage: two voxels per thread, one CTA per block (the range
    // is whole blocks)
    if (i32) {
      sparse_pair16<S, COLL><<<(unsigned)((a.s1 - a.s0) / E3), SP_THREADS, 0, s>>>(a);
      pair = true;
    }
  }
  if (pair) {
  } else if (MODE == MODE_INTERIOR && i32) {
    sparse_kernel<S, E, COLL, MODE, int32_t><<<nb, SP_THREADS, 0, s>>>(a);
  } else {
    sparse_kernel<S, E, COLL, MODE><<<nb, SP_THREADS, 0, s>>>(a);
  }
  prof_end(g, s, pr);
}

static bool fits_i32(const Level& L, int q) { return (int64_t)q * L.n_slots < ((int64_t)1 << 31); }


template <int S, int E, int COLL>
static lbm_status sparse_step_t(Grid& g, Level& L, cudaStream_t s) {
  constexpr int64_t E3 = (int64_t)E * E * E;
  SparseArgs a{};
  a.fin = L.f[L.cur];
  a.fout = L.f[L.cur ^ 1];
  a.nbr = L.nbr_d;
  a.flags = L.flags_d;
  a.wmask = L.wmask_d;
  a.blk_walls = L.blk_walls_d;
  a.omega = (float)(1.0 / g.phys.tau);
  if (g.phys.schedule == LBM_SCHEDULE_MONOLITHIC) {
    a.bc = L.bc_full_d;
    a.s0 = 0;
    a.s1 = L.n_blocks * E3;
    launch_range<S, E, COLL, MODE_MONOLITHIC>(g, a, s, "sparse_monolithic", L.n_updated);
  } else {
    // the two group kernels read the previous state and write disjoint
    // blocks: the boundary group's runs beside the interior one on the
    // grid's high-priority group stream
    const bool fork = L.n_b > 0 && L.n_b < L.n_blocks;
    cudaStream_t sb = s;
    if (fork) {
      lbm_status st = group_fork(g, s, &sb);
      if (st) return st;
    }
    if (L.bitmask) {
      a.bnd_bits = L.bnd_bits_d;
      a.bc_idx = L.bc_idx_d;
      a.bc_cmp = L.bc_cmp_d;
      a.s0 = 0;
      a.s1 = L.n_blocks * E3;
      launch_range<S, E, COLL, MODE_BOUNDARY_BM>(g, a, sb, "sparse_boundary_bitmask", L.n_upd_b);
      launch_range<S, E, COLL, MODE_INTERIOR_BM>(g, a, s, "sparse_interior_bitmask",
                                                 L.n_updated - L.n_upd_b);
    } else {
      a.bc = L.bc_grp_d;
      a.s0 = 0;
      a.s1 = L.n_b * E3;
      launch_range<S, E, COLL, MODE_BOUNDARY>(g, a, sb, "sparse_boundary", L.n_upd_b);
      a.s0 = L.n_b * E3;
      a.s1 = L.n_blocks * E3;
      bool staged = false;
      if constexpr (E == 8) {
        if (L.variant == VARIANT_STAGED) {
          launch_staged<S, COLL>(g, a, s, "sparse_interior_staged", L.n_updated - L.n_upd_b);
          staged = true;
        }
      }
      if (!staged)
        launch_range<S, E, COLL, MODE_INTERIOR>(g, a, s, "sparse_interior", L.n_updated - L.n_upd_b,
                                                fits_i32(L, Q));
    }
    if (fork) {
      lbm_status st = group_join(g, s);
      if (st) return st;
    }
  }
  LBM_CUDA(cudaGetLastError());
  L.cur ^= 1;
  return LBM_OK;
}

template <int S, int COLL>
static void uniform_range_t(Grid& g, Level& L, int64_t b0, int64_t b1, const void* fin, void* fout,
                            float omega, cudaStream_t s, const char* name, int64_t units) {
  SparseArgs a{};
  a.fin = fin;
  a.fout = fout;
  a.nbr = L.nbr_d;
  a.flags = L.flags_d;
  a.wmask = L.wmask_d;
  a.blk_walls = L.blk_walls_d;
  a.omega = omega;
  a.s0 = b0 * 512;
  a.s1 = b1 * 512;
  if (L.variant == VARIANT_STAGED) launch_staged<S, COLL>(g, a, s, name, units);
  else launch_range<S, 8, COLL, MODE_INTERIOR>(g, a, s, name, units, fits_i32(L, Q));
}

lbm_status sparse_reg_blocks(Grid& g, Level& L, const void* fin, void* fout, float omega,
                             cudaStream_t s, const char* name) {
  if (L.n_reg_blocks <= 0) return LBM_OK;
  const bool bgk = g.phys.collision == C_BGK;
  switch (g.phys.storage) {
    case S_F32:
      bgk ? reg_list_t<S_F32, C_BGK>(g, L, fin, fout, omega, s, name)
          : reg_list_t<S_F32, C_REG>(g, L, fin, fout, omega, s, name);
      break;
    case S_F16:
      bgk ? reg_list_t<S_F16, C_BGK>(g, L, fin, fout, omega, s, name)
          : reg_list_t<S_F16, C_REG>(g, L, fin, fout, omega, s, name);
      break;
    default:
      bgk ? reg_list_t<S_BF16, C_BGK>(g, L, fin, fout, omega, s, name)
          : reg_list_t<S_BF16, C_REG>(g, L, fin, fout, omega, s, name);
  }
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}

lbm_status sparse_uniform_range(Grid& g, Level& L, int64_t b0, int64_t b1, const void* fin,
                                void* fout, float omega, cudaStream_t s, const char* name,
                                int64_t units) {
  const bool bgk = g.phys.collision == C_BGK;
  switch (g.phys.storage) {
    case S_F32:
      bgk ? uniform_range_t<S_F32, C_BGK>(g, L, b0, b1, fin, fout, omega, s, name, units)
          : uniform_range_t<S_F32, C_REG>(g, L, b0, b1, fin, fout, omega, s, name, units);
      break;
    case S_F16:
      bgk ? uniform_range_t<S_F16, C_BGK>(g, L, b0, b1, fin, fout, omega, s, name, units)
          : uniform_range_t<S_F16, C_REG>(g, L, b0, b1, fin, fout, omega, s, name, units);
      break;
    default:
      bgk ? uniform_range_t<S_BF16, C_BGK>(g, L, b0, b1, fin, fout, omega, s, name, units)
          : uniform_range_t<S_BF16, C_REG>(g, L, b0, b1, fin, fout, omega, s, name, units);
  }
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}

template <int S, int E>
static lbm_status sparse_step_e(Grid& g, Level& L, cudaStream_t s) {
  return g.phys.collision == C_BGK ? sparse_step_t<S, E, C_BGK>(g, L, s)
                                   : sparse_step_t<S, E, C_REG>(g, L, s);
}

template <int S>
static lbm_status sparse_step_s(Grid& g, Level& L, cudaStream_t s) {
  return L.E == 8 ? sparse_step_e<S, 8>(g, L, s) : sparse_step_e<S, 4>(g, L, s);
}

lbm_status sparse_step(Grid& g, Level& L, cudaStream_t s) {
  switch (g.phys.storage) {
    case S_F32: return sparse_step_s<S_F32>(g, L, s);
    case S_F16: return sparse_step_s<S_F16>(g, L, s);
    default: return sparse_step_s<S_BF16>(g, L, s);
  }
}

}  // namespace LBM_LNS
}  // namespace lbm
