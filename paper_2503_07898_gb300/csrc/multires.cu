// multires.cu - multi-resolution grids: layout, interface kernels, schedule.
//
// Disaggregation of a multi-resolution grid (Sec. 5; Sec. 6.3):
//   definition     P_d, the distance of a voxel to a resolution jump; 0 means
//                  a D3Q19 neighbour belongs to another level.
//   classification per level, G_c = blocks holding a voxel at distance 0,
//                  G_i = all other blocks.
//   mapping        per level an 8^3-block sparse grid; G_c blocks first,
//                  then G_i, each in Morton order.
//   operations     inside G_c the grouping goes down to the voxel: the
//                  interface voxels (a pull read from another level) run
//                  mr_iface from a per-level list; every other voxel of the
//                  level runs the lean fused stream-collide kernel of the
//                  sparse grid (no cross-level data), kept off the interface
//                  voxels by a per-slot mask; on the learned closure's levels
//                  both run the network in the collision.  The unfused
//                  schedule streams whole blocks (mr_stream_split) and
//                  collides in a second pass (mr_collide).
//
// Time stepping (refinement factor 2, acoustic scaling): one step of level l
// contains two steps of level l-1.  Across a level jump the exchange is the
// level-(l-1) streaming of the two substeps, every level-l voxel being
// represented by 8 virtual subcells that hold its post-collision populations
// C at the start of its step and stream without colliding:
//   explosion   a level-(l-1) voxel pulling from a level-l region reads
//               C (substep 1) or, in substep 2, what that virtual subcell
//               received in substep 1: F0 (finer state at the step start)
//               when its source is a level-(l-1) voxel, else C;
//   coalescence a level-l voxel next to level l-1 pulls, per direction, the
//               mean of what its 8 subcells receive in substep 2: F1 (finer
//               state after substep 1) or the substep-1 value as above.
// Each non-coarsest level keeps a ring of three buffers, so F0 and F1 are
// still in memory when the coarser level coalesces: no copies.
//
// LBM_SCHEDULE_MONOLITHIC selects the unfused baseline of Sec. 6.3: at every
// level but the finest, all blocks run a stream kernel (pre-collision values
// to a scratch buffer) and then a collide kernel.  Both schedules perform the
// same arithmetic; in FP32 storage their results are bit-identical.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "d3q19.cuh"
#include "grid.h"
#include "closure.cuh"
#include "layout.h"
#include "sparse.cuh"

namespace lbm {
namespace LBM_LNS {

// ---------------------------------------------------------------- host layout

static inline int wrapi(int v, int n) { return ((v % n) + n) % n; }

// Directions whose pull from voxel l of block b leaves the level: the source
// block belongs to another level or, in a block next to a finer level
// (jump 1), a pull with two or three nonzero components crosses a face (or,
// for a corner direction, edge) neighbour block of another level, through
// which the subcells of the voxel trace.  mr_stream_split evaluates the same
// rule on the device.
static uint32_t mr_cross(const Level& V, int64_t b, int l) {
  const int lc[3] = {l & 7, (l >> 3) & 7, l >> 6};
  int e[3];
  for (int a = 0; a < 3; ++a) e[a] = lc[a] == 0 ? -1 : (lc[a] == 7 ? 1 : 0);
  const int32_t* nb = &V.nbr_h[(size_t)b * 27];
  auto at = [&](int dx, int dy, int dz) { return nb[13 + dx + 3 * dy + 9 * dz]; };
  const int jmp = V.jump_h[(size_t)b];
  uint32_t m = 0;
  for (int i = 1; i < Q; ++i) {
    const int c[3] = {cx(i), cy(i), cz(i)};
    bool k[3];
    int d[3], nnz = 0;
    for (int a = 0; a < 3; ++a) {
      k[a] = c[a] != 0 && e[a] == -c[a];
      d[a] = k[a] ? e[a] : 0;
      nnz += c[a] != 0;
    }
    bool plain = at(d[0], d[1], d[2]) >= 0;
    if (plain && jmp == 1 && nnz >= 2) {
      if ((k[0] && at(e[0], 0, 0) < 0) || (k[1] && at(0, e[1], 0) < 0) || (k[2] && at(0, 0, e[2]) < 0))
        plain = false;
      if (nnz == 3 && ((k[0] && k[1] && at(e[0], e[1], 0) < 0) || (k[0] && k[2] && at(e[0], 0, e[2]) < 0) ||
                       (k[1] && k[2] && at(0, e[1], e[2]) < 0)))
        plain = false;
    }
    if (!plain) m |= 1u << i;
  }
  return m;
}

// The interface voxels of a level (all in G_c blocks) in slot order.
static void mr_iface_list(Level& V) {
  V.iface_slot_h.clear();
  V.iface_cross_h.clear();
  for (int64_t b = 0; b < V.n_c; ++b)
    for (int l = 0; l < 512; ++l) {
      const uint32_t m = mr_cross(V, b, l);
      if (!m) continue;
      V.iface_slot_h.push_back((int32_t)(b * 512 + l));
      V.iface_cross_h.push_back(m);
    }
  V.n_iface = (int64_t)V.iface_slot_h.size();
}

// Mark the interface voxels in a per-slot lean-kernel mask (bit 31) and their
// blocks in the per-block mask bits.
static void mr_iface_masks(const Level& V, std::vector<uint32_t>& wm, std::vector<uint8_t>& bw) {
  for (int64_t k = 0; k < V.n_iface; ++k) {
    const int32_t sl = V.iface_slot_h[(size_t)k];
    wm[(size_t)sl] |= 1u << 31;
    bw[(size_t)(sl / 512)] = 1;
  }
}

static lbm_status mr_upload(Grid& g, void** dst, const void* src, size_t bytes) {
  g.dfree(*dst, g.stream);
  *dst = g.dalloc(bytes + 16, g.stream);
  if (!*dst) return fail(LBM_ERR_OOM, "device allocation failed");
  if (bytes) LBM_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return LBM_OK;
}

lbm_status multires_build(Grid& g, const int fin[3], int L, const uint8_t* lmap) {
  if (L < 1 || L > 4) return fail(LBM_ERR_INVALID, "n_levels must be 1..4");
  const int C = 8 << (L - 1);  // level-map cell (finest voxels) = coarsest block
  for (int a = 0; a < 3; ++a)
    if (fin[a] <= 0 || fin[a] % C) return fail(LBM_ERR_INVALID, "finest dims must be multiples of 8*2^(n_levels-1)");
  const int mx = fin[0] / C, my = fin[1] / C, mz = fin[2] / C;
  auto mapv = [&](int x, int y, int z) {
    return (int)lmap[wrapi(x, mx) + (size_t)mx * (wrapi(y, my) + (size_t)my * wrapi(z, mz))];
  };
  // walls and boundary nodes lie on the finest level: every map cell on a
  // non-periodic side is level 0, so coarser levels (and every explosion /
  // coalescence trace) stay at least one coarsest block from the walls and
  // the tables below may wrap as on a periodic box
  const int md[3] = {mx, my, mz};
  for (int a = 0; a < 3; ++a) {
    if (g.phys.periodic[a]) continue;
    for (int i = 0; i < md[(a + 1) % 3]; ++i)
      for (int j = 0; j < md[(a + 2) % 3]; ++j)
        for (int side = 0; side < 2; ++side) {
          int c[3];
          c[a] = side ? md[a] - 1 : 0;
          c[(a + 1) % 3] = i;
          c[(a + 2) % 3] = j;
          if (mapv(c[0], c[1], c[2]) != 0)
            return fail(LBM_ERR_UNSUPPORTED,
                        "map cells on a non-periodic side must be level 0 (walls on the finest level)");
        }
  }
  for (int z = 0; z < mz; ++z)
    for (int y = 0; y < my; ++y)
      for (int x = 0; x < mx; ++x) {
        const int lv = mapv(x, y, z);
        if (lv >= L) return fail(LBM_ERR_INVALID, "level map value >= n_levels");
        for (int k = 0; k < 27; ++k) {
          const int o = mapv(x + k % 3 - 1, y + (k / 3) % 3 - 1, z + k / 9 - 1);
          if (std::abs(o - lv) > 1) return fail(LBM_ERR_INVALID, "level map violates 2:1 grading");
        }
      }
  g.n_levels = L;
  // owner level of the level-l block (bx, by, bz)
  auto owner = [&](int l, int bx, int by, int bz) {
    const int s = (8 << l) ;  // block edge in finest voxels
    return mapv(bx * s / C - (bx * s < 0 ? 1 : 0), by * s / C - (by * s < 0 ? 1 : 0),
                bz * s / C - (bz * s < 0 ? 1 : 0));
  };
  // pass 1: per level active blocks, jump type, order, block maps
  for (int l = 0; l < L; ++l) {
    Level& V = g.lv[l];
    V.E = 8;
    V.nx = fin[0] >> l;
    V.ny = fin[1] >> l;
    V.nz = fin[2] >> l;
    V.nbx = V.nx / 8;
    V.nby = V.ny / 8;
    V.nbz = V.nz / 8;
    V.nbuf = 3;
    std::vector<int64_t> ids;
    std::vector<uint8_t> jt;
    const int64_t nvb = (int64_t)V.nbx * V.nby * V.nbz;
    std::vector<uint8_t> jump_v((size_t)nvb, 0);
    for (int64_t vb = 0; vb < nvb; ++vb) {
      const int bx = (int)(vb % V.nbx), by = (int)((vb / V.nbx) % V.nby),
                bz = (int)(vb / ((int64_t)V.nbx * V.nby));
      if (owner(l, bx, by, bz) != l) continue;
      int j = 0;
      for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        if (std::abs(dx) + std::abs(dy) + std::abs(dz) == 0 ||
            (Q == 19 && std::abs(dx) + std::abs(dy) + std::abs(dz) == 3))
          continue;  // D3Q19 reaches face and edge neighbours only, D3Q27 corners too
        const int o = owner(l, wrapi(bx + dx, V.nbx), wrapi(by + dy, V.nby), wrapi(bz + dz, V.nbz));
        if (o == l) continue;
        const int t = o < l ? 1 : 2;
        if (j && j != t) return fail(LBM_ERR_INVALID, "a block touches a finer and a coarser level");
        j = t;
      }
      jump_v[(size_t)vb] = (uint8_t)j;
      ids.push_back(vb);
    }
    auto key = [&](int64_t vb) {
      const uint32_t bx = (uint32_t)(vb % V.nbx), by = (uint32_t)((vb / V.nbx) % V.nby),
                     bz = (uint32_t)(vb / ((int64_t)V.nbx * V.nby));
      return ((uint64_t)(jump_v[(size_t)vb] ? 0 : 1) << 32) | morton3(bx, by, bz);
    };
    std::sort(ids.begin(), ids.end(), [&](int64_t a, int64_t b) { return key(a) < key(b); });
    V.n_blocks = (int64_t)ids.size();
    V.n_c = 0;
    V.bmap_h.assign((size_t)nvb, -1);
    V.coords_h.resize((size_t)V.n_blocks * 3);
    V.jump_h.resize((size_t)V.n_blocks);
    for (int64_t b = 0; b < V.n_blocks; ++b) {
      const int64_t vb = ids[(size_t)b];
      V.bmap_h[(size_t)vb] = (int32_t)b;
      V.coords_h[(size_t)b * 3 + 0] = (int32_t)(vb % V.nbx);
      V.coords_h[(size_t)b * 3 + 1] = (int32_t)((vb / V.nbx) % V.nby);
      V.coords_h[(size_t)b * 3 + 2] = (int32_t)(vb / ((int64_t)V.nbx * V.nby));
      V.jump_h[(size_t)b] = jump_v[(size_t)vb];
      if (jump_v[(size_t)vb]) ++V.n_c;
    }
    V.n_b = V.n_c;
    V.n_slots = V.n_blocks * 512;
    V.n_updated = V.n_slots;
  }
  // pass 2: neighbour tables (same level, coarser, finer)
  for (int l = 0; l < L; ++l) {
    Level& V = g.lv[l];
    V.nbr_h.assign((size_t)V.n_blocks * 27, -1);
    V.xnbr_coarse_h.assign((size_t)V.n_blocks * 27, -1);
    V.xnbr_fine_h.assign((size_t)V.n_blocks * 27 * 8, -1);
    for (int64_t b = 0; b < V.n_blocks; ++b)
      for (int k = 0; k < 27; ++k) {
        const int qx = wrapi(V.coords_h[b * 3] + k % 3 - 1, V.nbx);
        const int qy = wrapi(V.coords_h[b * 3 + 1] + (k / 3) % 3 - 1, V.nby);
        const int qz = wrapi(V.coords_h[b * 3 + 2] + k / 9 - 1, V.nbz);
        V.nbr_h[(size_t)b * 27 + k] = V.bmap_h[qx + (size_t)V.nbx * (qy + (size_t)V.nby * qz)];
        const int o = owner(l, qx, qy, qz);
        if (o == l + 1) {
          const Level& W = g.lv[l + 1];
          V.xnbr_coarse_h[(size_t)b * 27 + k] =
              W.bmap_h[(qx >> 1) + (size_t)W.nbx * ((qy >> 1) + (size_t)W.nby * (qz >> 1))];
        } else if (o == l - 1) {
          const Level& W = g.lv[l - 1];
          for (int j = 0; j < 8; ++j) {
            const int fx = 2 * qx + (j & 1), fy = 2 * qy + ((j >> 1) & 1), fz = 2 * qz + (j >> 2);
            V.xnbr_fine_h[((size_t)b * 27 + k) * 8 + j] =
                W.bmap_h[fx + (size_t)W.nbx * (fy + (size_t)W.nby * fz)];
          }
        }
      }
  }
  // pass 3: interface voxels
  for (int l = 0; l < L; ++l) mr_iface_list(g.lv[l]);
  return LBM_OK;
}

// Per-slot mask of the lean kernel (bit 31: the voxel is left to the
// interface kernel) and per-block mask bit, for every level; level 0 merges
// them with its walls in multires_set_boundary.  Uploads the interface lists.
lbm_status multires_finish(Grid& g) {
  for (int l = 0; l < g.n_levels; ++l) {
    Level& V = g.lv[l];
    std::vector<uint32_t> wm((size_t)V.n_slots, 0u);
    std::vector<uint8_t> bw((size_t)V.n_blocks, 0);
    mr_iface_masks(V, wm, bw);
    lbm_status st;
    if ((st = mr_upload(g, (void**)&V.wmask_d, wm.data(), wm.size() * 4)) ||
        (st = mr_upload(g, (void**)&V.blk_walls_d, bw.data(), bw.size())) ||
        (st = mr_upload(g, (void**)&V.iface_slot_d, V.iface_slot_h.data(), V.iface_slot_h.size() * 4)) ||
        (st = mr_upload(g, (void**)&V.iface_cross_d, V.iface_cross_h.data(), V.iface_cross_h.size() * 4)))
      return st;
  }
  return LBM_OK;
}

// Walls and boundary nodes of the finest level (Sec. 6.3's lid-driven
// cavity).  flags: level-0 virtual box; only voxels level 0 owns are read
// (solid, regularized velocity / pressure or fluid), and solid or
// regularized voxels must lie in G_i blocks (interface blocks run the
// interface kernel, which has no wall path).  Builds the per-slot flags, the
// wall mask (bit i = pull i bounces back: non-periodic box side or solid
// source; bit 30 regularized, bit 31 not updated), the per-block wall bit and
// the list of blocks holding regularized voxels, then the boundary values.
lbm_status multires_set_boundary(Grid& g, const uint8_t* flags, const float* bc_values,
                                 const float* def_bc) {
  Level& V = g.lv[0];
  const int nx = V.nx, ny = V.ny, nz = V.nz;
  const size_t nv = (size_t)nx * ny * nz;
  std::vector<uint8_t> fl(V.flags_h);
  if (flags) {
    for (size_t v = 0; v < nv; ++v) {
      if (flag_type(V.flags_h[v]) == T_OUTSIDE) continue;  // owned by another level
      const int t = flag_type(flags[v]);
      if (!type_updated(t) && t != T_SOLID)
        return fail(LBM_ERR_INVALID, "level-0 voxels must be fluid, solid or regularized");
      if (type_regularized(t) && flag_normal(flags[v]) > 5)
        return fail(LBM_ERR_INVALID, "regularized voxel with bad normal");
      fl[v] = flags[v];
    }
  }
  const int per[3] = {g.phys.periodic[0], g.phys.periodic[1], g.phys.periodic[2]};
  const int n3[3] = {nx, ny, nz};
  std::vector<uint8_t> sf((size_t)V.n_slots, (uint8_t)T_OUTSIDE);
  std::vector<uint32_t> wm((size_t)V.n_slots, 0u);
  std::vector<uint8_t> bw((size_t)V.n_blocks, 0);
  std::vector<int32_t> regb;
  int64_t n_upd = 0, n_reg = 0;
  for (int64_t b = 0; b < V.n_blocks; ++b) {
    bool has_reg = false;
    for (int l = 0; l < 512; ++l) {
      const int x = V.coords_h[b * 3] * 8 + (l & 7), y = V.coords_h[b * 3 + 1] * 8 + ((l >> 3) & 7),
                z = V.coords_h[b * 3 + 2] * 8 + (l >> 6);
      const uint8_t f = fl[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)];
      const int t = flag_type(f);
      sf[(size_t)(b * 512 + l)] = f;
      uint32_t m = 0;
      if (!type_updated(t)) m |= 1u << 31;
      if (type_regularized(t)) {
        m |= 1u << 30;
        has_reg = true;
        ++n_reg;
      }
      if (type_updated(t)) ++n_upd;
      for (int i = 1; i < Q; ++i) {
        int sc[3] = {x - cx(i), y - cy(i), z - cz(i)};
        bool wall = false;
        for (int a = 0; a < 3; ++a)
          if (sc[a] < 0 || sc[a] >= n3[a]) {
            if (per[a]) sc[a] = wrapi(sc[a], n3[a]);
            else wall = true;
          }
        if (!wall) wall = flag_type(fl[(size_t)sc[0] + (size_t)nx * ((size_t)sc[1] + (size_t)ny * sc[2])]) == T_SOLID;
        if (wall) m |= 1u << i;
      }
      wm[(size_t)(b * 512 + l)] = m;
      if (m) bw[(size_t)b] = 1;
    }
    if (bw[(size_t)b] && b < V.n_c)
      return fail(LBM_ERR_UNSUPPORTED, "walls and boundary nodes must lie in G_i blocks of level 0");
    if (has_reg) regb.push_back((int32_t)b);
  }
  // the interface voxels of the G_c blocks stay off the lean kernel
  mr_iface_masks(V, wm, bw);
  V.flags_h.swap(fl);
  V.n_updated = n_upd;
  V.n_reg = n_reg;
  V.n_reg_blocks = (int64_t)regb.size();
  lbm_status st;
  if ((st = mr_upload(g, (void**)&V.flags_d, sf.data(), sf.size())) ||
      (st = mr_upload(g, (void**)&V.wmask_d, wm.data(), wm.size() * 4)) ||
      (st = mr_upload(g, (void**)&V.blk_walls_d, bw.data(), bw.size())) ||
      (st = mr_upload(g, (void**)&V.reg_blocks_d, regb.data(), regb.size() * 4)))
    return st;
  return sparse_set_bc(g, V, bc_values, def_bc);
}

// ------------------------------------------------------------------ kernels

struct MrLv {
  int nx, ny, nz, nbx, nby;
  const int32_t* bmap;
};

struct MrArgs {
  MrLv me, co, fi;  // this level, coarser level, finer level
  const int32_t* nbr;
  const int32_t* coords;
  const uint8_t* jump;
  const void* cur;   // this level, start of this step
  const void* prev;  // this level, start of the coarser step (substep 2 explosion)
  void* out;
  const void* ccur;  // coarser level, start of its step
  const void* ff0;   // finer level at the start of this step
  const void* ff1;   // finer level after its first substep
  int k;             // 1 or 2: substep of this level inside the coarser step
  int64_t b0, b1;    // block range
  float omega;
  float tau;                  // relaxation time of this level (closure input)
  const ClosureParams* cp;    // learned closure (CLOSURE kernels only)
  int* status;
};

__device__ __forceinline__ int wrapd(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ bool mr_owns(const MrLv& v, int x, int y, int z) {
  return v.bmap[(x >> 3) + v.nbx * ((y >> 3) + v.nby * (z >> 3))] >= 0;
}

// Velocity components by runtime index: the interface rules below run for a
// few populations of a few voxels only, so they take the direction as a
// runtime value and exist once in the kernel instead of once per direction.
#if LBM_Q == 27
#define MR_ROW(f)                                                                        \
  {f(0), f(1), f(2), f(3), f(4), f(5), f(6), f(7), f(8), f(9), f(10), f(11), f(12), f(13), \
   f(14), f(15), f(16), f(17), f(18), f(19), f(20), f(21), f(22), f(23), f(24), f(25), f(26)}
#else
#define MR_ROW(f)                                                                        \
  {f(0), f(1), f(2), f(3), f(4), f(5), f(6), f(7), f(8), f(9), f(10), f(11), f(12), f(13), \
   f(14), f(15), f(16), f(17), f(18)}
#endif
__constant__ int8_t mr_c[3][Q] = {MR_ROW(cx), MR_ROW(cy), MR_ROW(cz)};
#undef MR_ROW

// Population i at a (wrapped) voxel of a level; a miss is an internal error
// (recorded, value 0) rather than an out-of-bounds access.
template <int S>
__device__ __forceinline__ float mr_load(const void* buf, const MrLv& v, int x, int y, int z, int i,
                                         int* status) {
  using T = typename Codec<S>::T;
  const int b = v.bmap[(x >> 3) + v.nbx * ((y >> 3) + v.nby * (z >> 3))];
  if (b < 0) {
    atomicExch(status, (int)LBM_ERR_INTERNAL);
    return 0.f;
  }
  const int64_t idx = ((int64_t)b * Q + i) * 512 + (x & 7) + 8 * ((y & 7) + 8 * (z & 7));
  return Codec<S>::load_rt(((const T*)buf)[idx], i);
}

// Explosion: this (finer) level pulls population i (velocity c) of voxel G
// from a coarser region.
template <int S>
__device__ __forceinline__ float explosion(const MrArgs& a, int i, int ccx, int ccy, int ccz,
                                           int gx, int gy, int gz) {
  const int qx = wrapd(gx - ccx, a.me.nx), qy = wrapd(gy - ccy, a.me.ny),
            qz = wrapd(gz - ccz, a.me.nz);
  if (a.k == 1) return mr_load<S>(a.ccur, a.co, qx >> 1, qy >> 1, qz >> 1, i, a.status);
  const int rx = wrapd(qx - ccx, a.me.nx), ry = wrapd(qy - ccy, a.me.ny),
            rz = wrapd(qz - ccz, a.me.nz);
  if (mr_owns(a.me, rx, ry, rz)) return mr_load<S>(a.prev, a.me, rx, ry, rz, i, a.status);
  return mr_load<S>(a.ccur, a.co, rx >> 1, ry >> 1, rz >> 1, i, a.status);
}

// Coalescence: this (coarser) level pulls population i of voxel G as the mean
// over its 8 subcells of what they receive in the second finer substep.
template <int S>
__device__ __forceinline__ float coalescence(const MrArgs& a, int i, int ccx, int ccy, int ccz,
                                             int gx, int gy, int gz) {
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int rx = wrapd(2 * gx + (j & 1) - ccx, a.fi.nx);
    const int ry = wrapd(2 * gy + ((j >> 1) & 1) - ccy, a.fi.ny);
    const int rz = wrapd(2 * gz + (j >> 2) - ccz, a.fi.nz);
    if (mr_owns(a.fi, rx, ry, rz)) {
      v[j] = mr_load<S>(a.ff1, a.fi, rx, ry, rz, i, a.status);
    } else {
      const int sx = wrapd(rx - ccx, a.fi.nx), sy = wrapd(ry - ccy, a.fi.ny),
                sz = wrapd(rz - ccz, a.fi.nz);
      v[j] = mr_owns(a.fi, sx, sy, sz)
                 ? mr_load<S>(a.ff0, a.fi, sx, sy, sz, i, a.status)
                 : mr_load<S>(a.cur, a.me, sx >> 1, sy >> 1, sz >> 1, i, a.status);
    }
  }
  // pairwise means along x, then y, then z (exact when the 8 values are equal)
  const float m0 = 0.5f * (v[0] + v[1]), m1 = 0.5f * (v[2] + v[3]);
  const float m2 = 0.5f * (v[4] + v[5]), m3 = 0.5f * (v[6] + v[7]);
  const float n0 = 0.5f * (m0 + m1), n1 = 0.5f * (m2 + m3);
  return 0.5f * (n0 + n1);
}

// Pre-collision scratch of the unfused schedule: shifted values stay raw FP32
// under FP32 storage (an exact round trip, so both schedules agree bit for
// bit); under 16-bit storage the scratch uses the storage type.
template <int S> struct TmpCodec {
  using T = typename Codec<S>::T;
  template <int I> __device__ static __forceinline__ float load(T v) {
    return Codec<S>::template load<I>(v);
  }
  template <int I> __device__ static __forceinline__ T store(float s) {
    return Codec<S>::template store<I>(s);
  }
};
template <> struct TmpCodec<S_F32> {
  using T = float;
  template <int I> __device__ static __forceinline__ float load(T v) { return v; }
  template <int I> __device__ static __forceinline__ T store(float s) { return s; }
};

// Stream pass of the unfused schedule (Sec. 6.3's baseline): every voxel of
// every block of the level pulls, explosion / coalescence included, and
// writes its pre-collision values to the scratch buffer; mr_collide follows.
template <int S>
__global__ void __launch_bounds__(256, Q == 27 ? 3 : 4) mr_stream_split(MrArgs a) {
  using T = typename Codec<S>::T;
  const int64_t b = a.b0 + blockIdx.x / 2;
  __shared__ float mr_slow[Q][256];  // per-thread values of pulls that leave the level
  if (b >= a.b1) return;  // uniform per CTA
  const int32_t* __restrict__ nbr = a.nbr + b * 27;
  const int l = (blockIdx.x & 1) * 256 + threadIdx.x;
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  const int ox = a.coords[b * 3] * 8, oy = a.coords[b * 3 + 1] * 8, oz = a.coords[b * 3 + 2] * 8;
  const int jmp = a.jump[b];
  const T* __restrict__ cur = (const T*)a.cur;
  // same-level pulls: the blocks a pull can enter are looked up once per
  // voxel (as in the sparse pull); a missing one means another level
  const int ex = lx == 0 ? -1 : (lx == 7 ? 1 : 0);
  const int ey = ly == 0 ? -1 : (ly == 7 ? 1 : 0);
  const int ez = lz == 0 ? -1 : (lz == 7 ? 1 : 0);
  const int bb = (int)b;
  const int nX = __ldg(nbr + 13 + ex), nY = __ldg(nbr + 13 + 3 * ey);
  const int nZ = __ldg(nbr + 13 + 9 * ez);
  const int nXY = __ldg(nbr + 13 + ex + 3 * ey), nXZ = __ldg(nbr + 13 + ex + 9 * ez);
  const int nYZ = __ldg(nbr + 13 + 3 * ey + 9 * ez);
  const int nXYZ = Q == 27 ? __ldg(nbr + 13 + ex + 3 * ey + 9 * ez) : bb;
  const int xp = (lx - 1) & 7, xn = (lx + 1) & 7;
  const int yp = ((ly - 1) & 7) * 8, yn = ((ly + 1) & 7) * 8, y0 = ly * 8;
  const int zp = ((lz - 1) & 7) * 64, zn = ((lz + 1) & 7) * 64, z0 = lz * 64;
  // the source block of pull I, and whether it lies on this level
  auto source = [&](auto ic, int& nb) -> bool {
    constexpr int I = decltype(ic)::value;
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    const bool kx = X != 0 && ex == -X;
    const bool ky = Y != 0 && ey == -Y;
    const bool kz = Z != 0 && ez == -Z;
    nb = bb;
    if constexpr (X != 0 && Y != 0 && Z != 0)
      nb = kz ? (kx ? (ky ? nXYZ : nXZ) : (ky ? nYZ : nZ)) : (kx ? (ky ? nXY : nX) : (ky ? nY : bb));
    else if constexpr (X != 0 && Y != 0) nb = kx ? (ky ? nXY : nX) : (ky ? nY : bb);
    else if constexpr (X != 0 && Z != 0) nb = kx ? (kz ? nXZ : nX) : (kz ? nZ : bb);
    else if constexpr (Y != 0 && Z != 0) nb = ky ? (kz ? nYZ : nY) : (kz ? nZ : bb);
    else if constexpr (X != 0) nb = kx ? nX : bb;
    else if constexpr (Y != 0) nb = ky ? nY : bb;
    else if constexpr (Z != 0) nb = kz ? nZ : bb;
    bool plain = nb >= 0;
    if constexpr ((X != 0) + (Y != 0) + (Z != 0) >= 2) {
      // a coarse voxel's subcells also trace through the face (and, for a
      // corner direction, edge) neighbours the pull crosses; all of them
      // must be on this level
      if (plain && jmp == 1) {
        if (kx && nX < 0) plain = false;
        if (ky && nY < 0) plain = false;
        if (kz && nZ < 0) plain = false;
        if constexpr ((X != 0) + (Y != 0) + (Z != 0) == 3) {
          if (kx && ky && nXY < 0) plain = false;
          if (kx && kz && nXZ < 0) plain = false;
          if (ky && kz && nYZ < 0) plain = false;
        }
      }
    }
    return plain;
  };
  // 1. directions whose pull leaves the level
  uint32_t cross = 0u;
  static_for<Q>([&](auto ic) {
    int nb;
    if (!source(ic, nb)) cross |= 1u << decltype(ic)::value;
  });
  // 2. their values by explosion (from the coarser level) or coalescence
  // (from the finer one).  Only the voxels on a block face next to another
  // level have such pulls, so the (voxel, direction) pairs of the whole CTA
  // are listed and spread over all its threads: each pair is a chain of
  // dependent lookups, and one lane working through its own five or more
  // would hold up the CTA.  The values are parked in the owning thread's
  // column of shared memory, so no population is live across the loop.
  __shared__ uint16_t mr_work[256 * (Q - 1)];  // (thread << 5) | direction
  __shared__ int mr_wcount[8];
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = __popc(cross);
    int incl = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) mr_wcount[warp] = incl;
    __syncthreads();
    int pos = incl - n, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int c = mr_wcount[w];
      pos += w < warp ? c : 0;
      total += c;
    }
    for (uint32_t m = cross; m; m &= m - 1) mr_work[pos++] = (uint16_t)((threadIdx.x << 5) | (__ffs(m) - 1));
    if (total > 0) {  // uniform per CTA
      __syncthreads();
      for (int e = threadIdx.x; e < total; e += 256) {
        const int w = mr_work[e];
        const int t = w >> 5, i = w & 31;
        const int tl = (blockIdx.x & 1) * 256 + t;
        const int gx = ox + (tl & 7), gy = oy + ((tl >> 3) & 7), gz = oz + (tl >> 6);
        const int ccx = mr_c[0][i], ccy = mr_c[1][i], ccz = mr_c[2][i];
        mr_slow[i][t] = jmp == 2 ? explosion<S>(a, i, ccx, ccy, ccz, gx, gy, gz)
                                 : coalescence<S>(a, i, ccx, ccy, ccz, gx, gy, gz);
      }
      __syncthreads();
    }
  }
  // 3. the same-level pulls
  float g[Q];
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    int nb;
    source(ic, nb);
    if ((cross >> I) & 1u) {
      g[I] = mr_slow[I][threadIdx.x];
    } else {
      const int ls = (X > 0 ? xp : (X < 0 ? xn : lx)) + (Y > 0 ? yp : (Y < 0 ? yn : y0)) +
                     (Z > 0 ? zp : (Z < 0 ? zn : z0));
      g[I] = Codec<S>::template load<I>(cur[(int64_t)nb * (Q * 512) + (I * 512 + ls)]);
    }
  });
  using TT = typename TmpCodec<S>::T;
  TT* __restrict__ out = (TT*)a.out;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    out[(b * Q + I) * 512 + l] = TmpCodec<S>::template store<I>(g[I]);
  });
}

// The learned closure's relaxation rate for this thread's voxel: features of
// its pulled populations, then the network over the warp's 32 voxels (warp-
// collective: every lane takes part).  The populations wait in the thread's
// column of `park` meanwhile (volatile: the copies must really leave the
// registers, which the network needs).
// m receives the moments of g (rho - 1, j) for the collision.
__device__ __forceinline__ float closure_omega(float g[Q], float tau, ClosureCta* sm,
                                               float (*park)[256], float m[4]) {
  float x[MLP_IN];
  closure_features(g, tau, x, m);
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    *(volatile float*)&park[I][threadIdx.x] = g[I];
  });
  const float dtau = mlp_bf16_warp(x, sm->w, sm->stage[threadIdx.x >> 5]);
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    g[I] = *(volatile float*)&park[I][threadIdx.x];
  });
  return 1.f / fmaxf(tau + dtau, TAU_MIN);
}

// Lean step of a closure level: every non-interface voxel of the level pulls
// as in the sparse lean kernel, and the closure runs in the collision.  The
// masked voxels (interface voxels, bit 31) take part in the network with the
// rest state, so its warps stay full, and store nothing.
template <int S, int COLL, class IDX>
__global__ void __launch_bounds__(256, 3)
    mr_lean_closure(const void* fin, void* fout, const int32_t* __restrict__ nbr,
                    const uint32_t* __restrict__ wmask, const uint8_t* __restrict__ blk_walls,
                    float tau, const ClosureParams* cp) {
  using T = typename Codec<S>::T;
  extern __shared__ __align__(16) unsigned char mr_dyn_smem[];
  __shared__ float park[Q][256];
  ClosureCta* sm = reinterpret_cast<ClosureCta*>(mr_dyn_smem);
  closure_load_smem(sm->w, cp);
  __syncthreads();
  const int64_t slot = (int64_t)blockIdx.x * 256 + threadIdx.x;  // whole blocks: always a slot
  const int64_t b = slot >> 9;
  const int l = (int)(slot & 511);
  const bool walls = blk_walls[b] != 0;
  const uint32_t wm = walls ? wmask[slot] : 0u;
  const bool act = !(wm & 0xC0000000u);
  float g[Q];
  if (act) {
    sparse_pull_voxel<S, 8, IDX>((const T*)fin, nbr + b * 27, wm, b, l, walls, g);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = 0.f;
  }
  float m[4];
  const float omega = closure_omega(g, tau, sm, park, m);
  if (!act) return;
  collide_m<COLL>(g, omega, m[0], m[1], m[2], m[3]);
  T* __restrict__ out = (T*)fout;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    out[(b * Q + I) * 512 + l] = Codec<S>::template store<I>(g[I]);
  });
}

// Pull of one interface voxel (slot, bit set of its cross-level
// populations): explosion / coalescence values first, parked in the thread's
// column of `slow`, then the same-level pulls through the hoisted neighbour
// blocks.
template <int S>
__device__ __forceinline__ void mr_iface_pull(const MrArgs& a, int slot, uint32_t cross,
                                              float (*slow)[256], float g[Q]) {
  using T = typename Codec<S>::T;
  const int b = slot >> 9, l = slot & 511;
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  const int jmp = a.jump[b];
  {
    const int gx = a.coords[b * 3] * 8 + lx, gy = a.coords[b * 3 + 1] * 8 + ly,
              gz = a.coords[b * 3 + 2] * 8 + lz;
    for (uint32_t m = cross; m; m &= m - 1) {
      const int i = __ffs(m) - 1;
      const int ccx = mr_c[0][i], ccy = mr_c[1][i], ccz = mr_c[2][i];
      slow[i][threadIdx.x] = jmp == 2 ? explosion<S>(a, i, ccx, ccy, ccz, gx, gy, gz)
                                      : coalescence<S>(a, i, ccx, ccy, ccz, gx, gy, gz);
    }
  }
  const int32_t* __restrict__ nbr = a.nbr + (int64_t)b * 27;
  const int ex = lx == 0 ? -1 : (lx == 7 ? 1 : 0);
  const int ey = ly == 0 ? -1 : (ly == 7 ? 1 : 0);
  const int ez = lz == 0 ? -1 : (lz == 7 ? 1 : 0);
  const int nX = __ldg(nbr + 13 + ex), nY = __ldg(nbr + 13 + 3 * ey);
  const int nZ = __ldg(nbr + 13 + 9 * ez);
  const int nXY = __ldg(nbr + 13 + ex + 3 * ey), nXZ = __ldg(nbr + 13 + ex + 9 * ez);
  const int nYZ = __ldg(nbr + 13 + 3 * ey + 9 * ez);
  const int nXYZ = Q == 27 ? __ldg(nbr + 13 + ex + 3 * ey + 9 * ez) : b;
  const int xp = (lx - 1) & 7, xn = (lx + 1) & 7;
  const int yp = ((ly - 1) & 7) * 8, yn = ((ly + 1) & 7) * 8, y0 = ly * 8;
  const int zp = ((lz - 1) & 7) * 64, zn = ((lz + 1) & 7) * 64, z0 = lz * 64;
  const T* __restrict__ cur = (const T*)a.cur;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    if ((cross >> I) & 1u) {
      g[I] = slow[I][threadIdx.x];
    } else {
      const bool kx = X != 0 && ex == -X, ky = Y != 0 && ey == -Y, kz = Z != 0 && ez == -Z;
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
      g[I] = Codec<S>::template load<I>(cur[(int64_t)nb * (Q * 512) + (I * 512 + ls)]);
    }
  });
}

// Interface voxels of the fused schedule, one thread each (the list holds
// only voxels with a pull that leaves the level; the lean kernel updates the
// rest of their blocks).  CLOSURE: the learned closure in the collision;
// threads past the end of the list take part in the network (warp-
// collective, one call site) with the rest state and store nothing.
template <int S, int COLL, bool CLOSURE = false>
__global__ void __launch_bounds__(256, CLOSURE ? 3 : (Q == 27 ? 3 : 4))
    mr_iface(MrArgs a, const int32_t* __restrict__ slots, const uint32_t* __restrict__ crosses,
             int n) {
  using T = typename Codec<S>::T;
  extern __shared__ __align__(16) unsigned char mr_dyn_smem[];
  __shared__ float mr_slow[Q][256];
  if constexpr (CLOSURE) {
    closure_load_smem(reinterpret_cast<ClosureCta*>(mr_dyn_smem)->w, a.cp);
    __syncthreads();
  }
  const int t = blockIdx.x * 256 + threadIdx.x;
  const bool act = t < n;
  if constexpr (!CLOSURE) {
    if (!act) return;
  }
  int slot = 0;
  float g[Q];
  if (act) {
    slot = slots[t];
    mr_iface_pull<S>(a, slot, crosses[t], mr_slow, g);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = 0.f;
  }
  float omega = a.omega;
  float m[4];
  if constexpr (CLOSURE)
    omega = closure_omega(g, a.tau, reinterpret_cast<ClosureCta*>(mr_dyn_smem), mr_slow, m);
  if (!act) return;
  if constexpr (CLOSURE) collide_m<COLL>(g, omega, m[0], m[1], m[2], m[3]);
  else collide<COLL>(g, omega);
  const int b = slot >> 9, l = slot & 511;
  T* __restrict__ out = (T*)a.out;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    out[((int64_t)b * Q + I) * 512 + l] = Codec<S>::template store<I>(g[I]);
  });
}

// Unfused baseline: collision of the pre-collision values written by the
// split stream kernel.
template <int S, int COLL>
__global__ void __launch_bounds__(256) mr_collide(const void* tmp, void* out, int64_t b0,
                                                  int64_t b1, float omega) {
  using T = typename Codec<S>::T;
  const int64_t b = b0 + blockIdx.x / 2;
  if (b >= b1) return;
  const int l = (blockIdx.x & 1) * 256 + threadIdx.x;
  using TT = typename TmpCodec<S>::T;
  const TT* in = (const TT*)tmp;
  float g[Q];
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    g[I] = TmpCodec<S>::template load<I>(in[(b * Q + I) * 512 + l]);
  });
  collide<COLL>(g, omega);
  T* o = (T*)out;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    o[(b * Q + I) * 512 + l] = Codec<S>::template store<I>(g[I]);
  });
}

// ----------------------------------------------------------------- schedule

static MrLv view(const Level& V) {
  MrLv m;
  m.nx = V.nx;
  m.ny = V.ny;
  m.nz = V.nz;
  m.nbx = V.nbx;
  m.nby = V.nby;
  m.bmap = V.bmap_d;
  return m;
}

static const char* kname(int kind, int l) {
  static const char* names[4][4] = {
      {"mr_uniform_l0", "mr_uniform_l1", "mr_uniform_l2", "mr_uniform_l3"},
      {"mr_iface_l0", "mr_iface_l1", "mr_iface_l2", "mr_iface_l3"},
      {"mr_stream_split_l0", "mr_stream_split_l1", "mr_stream_split_l2", "mr_stream_split_l3"},
      {"mr_collide_l0", "mr_collide_l1", "mr_collide_l2", "mr_collide_l3"}};
  return names[kind][l];
}

template <int S, int COLL>
static lbm_status mr_advance(Grid& g, int l, int k, cudaStream_t s) {
  Level& V = g.lv[l];
  const double tau_l = 0.5 + (g.phys.tau - 0.5) / (double)(1 << l);
  const float omega = (float)(1.0 / tau_l);
  const int c = V.cur, nx = (c + 1) % 3, pv = (c + 2) % 3;
  const bool unfused = g.phys.schedule == LBM_SCHEDULE_MONOLITHIC && l > 0;
  const bool closure = g.phys.closure && g.closure_loaded && l > 0;
  const size_t csm = closure ? sizeof(ClosureCta) : 0;
  lbm_status st;
  MrArgs a{};
  a.me = view(V);
  a.nbr = V.nbr_d;
  a.coords = V.coords_d;
  a.jump = V.jump_d;
  a.cur = V.f[c];
  a.prev = V.f[pv];
  a.k = k;
  a.omega = omega;
  a.tau = (float)tau_l;
  a.cp = (const ClosureParams*)g.closure_d;
  a.status = g.status_d;
  if (l + 1 < g.n_levels) {
    const Level& W = g.lv[l + 1];
    a.co = view(W);
    a.ccur = W.f[W.cur];
  }
  // Fused schedule: every voxel without a cross-level pull (all of G_i and
  // most of G_c) runs the lean kernel, which needs no cross-level data and
  // shares no output with the interface voxels: launched first, on the
  // level's second stream, it overlaps the finer substeps and this level's
  // interface launch; joined before returning.  It waits only for this
  // level's previous step (mr_fork, recorded when it completed), so it also
  // overlaps the coarser levels' interface launches that run between two
  // steps of this level.  Those read this level's ring buffers only at its
  // interface voxels (next to another level), which the lean kernel never
  // writes.  On closure levels both kernels run the network in the collision.
  const bool fork = !unfused && V.n_blocks > 0;
  const cudaStream_t s_main = s;
  if (fork) {
    LBM_CUDA(cudaStreamWaitEvent(g.mr_aux[l], g.mr_fork[l], 0));
    s = g.mr_aux[l];
    if (closure) {
      const int pr = prof_begin(g, s, kname(0, l), V.n_updated - V.n_iface);
      // 32-bit element offsets in the pull while the level's Q 512 n_blocks
      // elements fit in 31 bits
      if ((int64_t)Q * 512 * V.n_blocks < (1LL << 31))
        mr_lean_closure<S, COLL, int32_t><<<(unsigned)(2 * V.n_blocks), 256, csm, s>>>(
            V.f[c], V.f[nx], V.nbr_d, V.wmask_d, V.blk_walls_d, (float)tau_l, a.cp);
      else
        mr_lean_closure<S, COLL, int64_t><<<(unsigned)(2 * V.n_blocks), 256, csm, s>>>(
            V.f[c], V.f[nx], V.nbr_d, V.wmask_d, V.blk_walls_d, (float)tau_l, a.cp);
      prof_end(g, s, pr);
    } else {
      st = sparse_uniform_range(g, V, 0, V.n_blocks, V.f[c], V.f[nx], omega, s, kname(0, l),
                                V.n_updated - V.n_iface - V.n_reg);
      if (st) return st;
      // regularized boundary voxels (a lid on level 0, in G_i blocks)
      if ((st = sparse_reg_blocks(g, V, V.f[c], V.f[nx], omega, s, "mr_regularized_l0"))) return st;
    }
    LBM_CUDA(cudaEventRecord(g.mr_join[l], s));
    s = s_main;
  }
  if (l > 0) {
    if ((st = mr_advance<S, COLL>(g, l - 1, 1, s))) return st;
    if ((st = mr_advance<S, COLL>(g, l - 1, 2, s))) return st;
  }
  if (l > 0) {
    const Level& W = g.lv[l - 1];
    a.fi = view(W);
    a.ff1 = W.f[(W.cur + 2) % 3];
    a.ff0 = W.f[(W.cur + 1) % 3];
  }
  if (unfused) {
    a.b0 = 0;
    a.b1 = V.n_blocks;
    a.out = V.tmp;
    if (V.n_blocks > 0) {
      const unsigned nb = (unsigned)(2 * V.n_blocks);
      int pr = prof_begin(g, s, kname(2, l), V.n_blocks * 512);
      mr_stream_split<S><<<nb, 256, 0, s>>>(a);
      prof_end(g, s, pr);
      pr = prof_begin(g, s, kname(3, l), V.n_blocks * 512);
      mr_collide<S, COLL><<<nb, 256, 0, s>>>(V.tmp, V.f[nx], 0, V.n_blocks, omega);
      prof_end(g, s, pr);
    }
  } else if (V.n_iface > 0) {
    a.out = V.f[nx];
    const unsigned nb = (unsigned)((V.n_iface + 255) / 256);
    const int pr = prof_begin(g, s, kname(1, l), V.n_iface);
    if (closure)
      mr_iface<S, COLL, true><<<nb, 256, csm, s>>>(a, V.iface_slot_d, V.iface_cross_d, (int)V.n_iface);
    else
      mr_iface<S, COLL><<<nb, 256, 0, s>>>(a, V.iface_slot_d, V.iface_cross_d, (int)V.n_iface);
    prof_end(g, s, pr);
  }
  LBM_CUDA(cudaGetLastError());
  if (fork) {
    LBM_CUDA(cudaStreamWaitEvent(s, g.mr_join[l], 0));
    LBM_CUDA(cudaEventRecord(g.mr_fork[l], s));
  }
  V.cur = nx;
  return LBM_OK;
}

lbm_status multires_step(Grid& g, cudaStream_t s, bool first) {
  const int top = g.n_levels - 1;
  if (g.phys.closure && !g.closure_loaded)
    return fail(LBM_ERR_INVALID, "closure enabled but no weights loaded (lbm_closure_load)");
  if (g.phys.closure && g.phys.schedule == LBM_SCHEDULE_MONOLITHIC)
    return fail(LBM_ERR_UNSUPPORTED, "the closure runs with the disaggregated schedule");
  if (g.phys.schedule == LBM_SCHEDULE_MONOLITHIC) {
    for (int l = 1; l < g.n_levels; ++l) {
      Level& V = g.lv[l];
      if (!V.tmp && V.n_blocks > 0) {
        V.tmp = g.dalloc(V.pop_bytes, s);
        if (!V.tmp) return fail(LBM_ERR_OOM, "unfused scratch allocation failed");
      }
    }
  }
  if (!g.mr_hi) {
    int least = 0, greatest = 0;
    LBM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    LBM_CUDA(cudaStreamCreateWithPriority(&g.mr_hi, cudaStreamNonBlocking, greatest));
    LBM_CUDA(cudaEventCreateWithFlags(&g.mr_in, cudaEventDisableTiming));
    LBM_CUDA(cudaEventCreateWithFlags(&g.mr_out, cudaEventDisableTiming));
  }
  // the coarse steps of one lbm_step call follow everything already on s;
  // between them only the level streams order the work
  if (first) {
    LBM_CUDA(cudaEventRecord(g.mr_in, s));
    LBM_CUDA(cudaStreamWaitEvent(g.mr_hi, g.mr_in, 0));
  }
  for (int l = 0; l < g.n_levels; ++l) {
    if (!g.mr_aux[l]) LBM_CUDA(cudaStreamCreateWithFlags(&g.mr_aux[l], cudaStreamNonBlocking));
    if (!g.mr_fork[l]) LBM_CUDA(cudaEventCreateWithFlags(&g.mr_fork[l], cudaEventDisableTiming));
    if (!g.mr_join[l]) LBM_CUDA(cudaEventCreateWithFlags(&g.mr_join[l], cudaEventDisableTiming));
    if (first) LBM_CUDA(cudaEventRecord(g.mr_fork[l], g.mr_hi));
  }
  // G_c launches on the high-priority stream: the scheduler hands them SMs
  // ahead of the bandwidth-bound G_i launches they overlap
  const cudaStream_t h = g.mr_hi;
  const bool bgk = g.phys.collision == C_BGK;
  lbm_status st;
  switch (g.phys.storage) {
    case S_F32: st = bgk ? mr_advance<S_F32, C_BGK>(g, top, 1, h) : mr_advance<S_F32, C_REG>(g, top, 1, h); break;
    case S_F16: st = bgk ? mr_advance<S_F16, C_BGK>(g, top, 1, h) : mr_advance<S_F16, C_REG>(g, top, 1, h); break;
    default: st = bgk ? mr_advance<S_BF16, C_BGK>(g, top, 1, h) : mr_advance<S_BF16, C_REG>(g, top, 1, h);
  }
  if (st) return st;
  LBM_CUDA(cudaEventRecord(g.mr_out, h));
  LBM_CUDA(cudaStreamWaitEvent(s, g.mr_out, 0));
  return LBM_OK;
}

}  // namespace LBM_LNS
}  // namespace lbm
