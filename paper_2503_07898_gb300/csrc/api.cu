// api.cu - C ABI entry points of liblbm (declared in include/lbm.h).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "d3q19.cuh"
#include "grid.h"
#include "layout.h"

namespace lbm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
lbm_status fail(lbm_status s, const std::string& msg) {
  set_error(msg);
  return s;
}
lbm_status cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
            ") in " + where);
  return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

void* Grid::dalloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (have_alloc) return alloc.alloc(alloc.ctx, bytes, (void*)s);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void Grid::dfree(void* p, cudaStream_t s) {
  if (!p) return;
  if (have_alloc) alloc.free(alloc.ctx, p, (void*)s);
  else cudaFree(p);
}

int prof_begin(Grid& g, cudaStream_t s, const char* name, int64_t units) {
  if (!g.prof) return -1;
  int k = -1;
  for (size_t i = 0; i < g.prof_names.size(); ++i)
    if (g.prof_names[i] == name) k = (int)i;
  if (k < 0) {
    g.prof_names.push_back(name);
    k = (int)g.prof_names.size() - 1;
  }
  ProfRec r{k, nullptr, nullptr, units};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  cudaEventRecord(r.a, s);
  g.prof_recs.push_back(r);
  return (int)g.prof_recs.size() - 1;
}

void prof_end(Grid& g, cudaStream_t s, int rec) {
  if (rec < 0) return;
  cudaEventRecord(g.prof_recs[(size_t)rec].b, s);
}

lbm_status group_fork(Grid& g, cudaStream_t s, cudaStream_t* hi) {
  if (!g.grp_hi) {
    int least = 0, greatest = 0;
    LBM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    LBM_CUDA(cudaStreamCreateWithPriority(&g.grp_hi, cudaStreamNonBlocking, greatest));
  }
  if (!g.grp_fork) LBM_CUDA(cudaEventCreateWithFlags(&g.grp_fork, cudaEventDisableTiming));
  if (!g.grp_join) LBM_CUDA(cudaEventCreateWithFlags(&g.grp_join, cudaEventDisableTiming));
  LBM_CUDA(cudaEventRecord(g.grp_fork, s));
  LBM_CUDA(cudaStreamWaitEvent(g.grp_hi, g.grp_fork, 0));
  *hi = g.grp_hi;
  return LBM_OK;
}

lbm_status group_join(Grid& g, cudaStream_t s) {
  LBM_CUDA(cudaEventRecord(g.grp_join, g.grp_hi));
  LBM_CUDA(cudaStreamWaitEvent(s, g.grp_join, 0));
  return LBM_OK;
}

void prof_clear(Grid& g) {
  for (auto& r : g.prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g.prof_recs.clear();
  g.prof_names.clear();
}

// RAII scratch allocation through the grid's allocator.
// Device address of a page-locked, mapped host array, or null (pageable or
// unregistered memory, or a null pointer).
template <class T> static T* mapped_host(T* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA-known pointer: clear the error
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<T*>(a.devicePointer);
}

struct Scratch {
  Grid& g;
  cudaStream_t s;
  void* p = nullptr;
  Scratch(Grid& g_, size_t bytes, cudaStream_t s_) : g(g_), s(s_) { p = g.dalloc(bytes, s); }
  ~Scratch() {
    if (p) {
      cudaStreamSynchronize(s);
      g.dfree(p, s);
    }
  }
};

static void free_level(Grid& g, Level& L) {
  cudaStream_t s = g.stream;
  g.dfree(L.f[0], s);
  g.dfree(L.f[1], s);
  g.dfree(L.f[2], s);
  g.dfree(L.tmp, s);
  g.dfree(L.jump_d, s);
  g.dfree(L.coords_d, s);
  g.dfree(L.flags_d, s);
  g.dfree(L.wmask_d, s);
  g.dfree(L.reg_list_d, s);
  g.dfree(L.bc_grp_d, s);
  g.dfree(L.bc_full_d, s);
  g.dfree(L.nbr_d, s);
  g.dfree(L.bmap_d, s);
  g.dfree(L.blk_walls_d, s);
  g.dfree(L.bnd_bits_d, s);
  g.dfree(L.reg_blocks_d, s);
  g.dfree(L.iface_slot_d, s);
  g.dfree(L.iface_cross_d, s);
  g.dfree(L.bc_idx_d, s);
  g.dfree(L.bc_cmp_d, s);
  L = Level();
}

static void free_grid(Grid& g) {
  cudaStreamSynchronize(g.stream);
  prof_clear(g);
  for (int l = 0; l < 4; ++l) {
    if (g.mr_aux[l]) {
      cudaStreamSynchronize(g.mr_aux[l]);
      cudaStreamDestroy(g.mr_aux[l]);
    }
    if (g.mr_fork[l]) cudaEventDestroy(g.mr_fork[l]);
    if (g.mr_join[l]) cudaEventDestroy(g.mr_join[l]);
    g.mr_aux[l] = nullptr;
    g.mr_fork[l] = g.mr_join[l] = nullptr;
  }
  if (g.mr_hi) {
    cudaStreamSynchronize(g.mr_hi);
    cudaStreamDestroy(g.mr_hi);
  }
  if (g.mr_in) cudaEventDestroy(g.mr_in);
  if (g.mr_out) cudaEventDestroy(g.mr_out);
  g.mr_hi = nullptr;
  g.mr_in = g.mr_out = nullptr;
  if (g.grp_hi) {
    cudaStreamSynchronize(g.grp_hi);
    cudaStreamDestroy(g.grp_hi);
  }
  if (g.grp_fork) cudaEventDestroy(g.grp_fork);
  if (g.grp_join) cudaEventDestroy(g.grp_join);
  g.grp_hi = nullptr;
  g.grp_fork = g.grp_join = nullptr;
  if (g.stream_ev) cudaEventDestroy(g.stream_ev);
  g.stream_ev = nullptr;
  for (int l = 0; l < 4; ++l) free_level(g, g.lv[l]);
  g.dfree(g.status_d, g.stream);
  g.dfree(g.partials_d, g.stream);
  g.dfree(g.sums_d, g.stream);
  g.dfree(g.closure_d, g.stream);
  g.closure_d = nullptr;
  g.status_d = nullptr;
  g.partials_d = nullptr;
  g.sums_d = nullptr;
}

static size_t storage_bytes(int storage) { return storage == LBM_STORAGE_F32 ? 4 : 2; }

static lbm_status check_physics(const lbm_physics* p) {
  if (!p) return fail(LBM_ERR_INVALID, "physics is NULL");
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(LBM_ERR_INVALID, "tau must be > 0.5");
  if (p->collision != LBM_COLLISION_BGK && p->collision != LBM_COLLISION_REG)
    return fail(LBM_ERR_INVALID, "unknown collision");
  if (p->storage < LBM_STORAGE_F32 || p->storage > LBM_STORAGE_BF16)
    return fail(LBM_ERR_INVALID, "unknown storage");
  if (p->schedule != LBM_SCHEDULE_DISAGGREGATED && p->schedule != LBM_SCHEDULE_MONOLITHIC &&
      p->schedule != LBM_SCHEDULE_BITMASK)
    return fail(LBM_ERR_INVALID, "unknown schedule");
  if (p->closure != 0 && p->closure != 1) return fail(LBM_ERR_INVALID, "closure must be 0 or 1");
  if (p->lattice != 0 && p->lattice != 19 && p->lattice != 27)
    return fail(LBM_ERR_INVALID, "lattice must be 19 or 27");
  if (p->lattice == 27 && p->closure)
    return fail(LBM_ERR_UNSUPPORTED, "the closure runs on D3Q19 grids");
  return LBM_OK;
}

template <class T>
static lbm_status upload(Grid& g, T** dst, const T* src, size_t count) {
  *dst = (T*)g.dalloc(count * sizeof(T), g.stream);
  if (!*dst) return fail(LBM_ERR_OOM, "device allocation failed");
  if (count) LBM_CUDA(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, g.stream));
  return LBM_OK;
}

static lbm_status alloc_common(Grid& g) {
  g.status_d = (int*)g.dalloc(sizeof(int), g.stream);
  g.partials_d = (double*)g.dalloc(sizeof(double) * 4 * kRedCtas * g.n_levels, g.stream);
  g.sums_d = (double*)g.dalloc(sizeof(double) * 4, g.stream);
  if (!g.status_d || !g.partials_d || !g.sums_d) return fail(LBM_ERR_OOM, "device allocation failed");
  LBM_CUDA(cudaMemsetAsync(g.status_d, 0, sizeof(int), g.stream));
  return LBM_OK;
}

static lbm_status alloc_populations(Grid& g, Level& L) {
  L.pop_bytes = (size_t)g.q * (size_t)L.n_slots * storage_bytes(g.phys.storage);
  for (int k = 0; k < L.nbuf; ++k) {
    L.f[k] = g.dalloc(L.pop_bytes, g.stream);
    if (!L.f[k]) return fail(LBM_ERR_OOM, "population buffer allocation failed");
    LBM_CUDA(cudaMemsetAsync(L.f[k], 0, L.pop_bytes, g.stream));
  }
  return LBM_OK;
}

static lbm_status begin(lbm_grid** out, const lbm_physics* phys, const lbm_allocator* alloc,
                        void* stream, Grid*& gp) {
  if (!out) return fail(LBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  lbm_status st = check_physics(phys);
  if (st) return st;
  if (alloc && (!alloc->alloc || !alloc->free))
    return fail(LBM_ERR_INVALID, "allocator needs alloc and free");
  lbm_grid* h = new (std::nothrow) lbm_grid();
  if (!h) return fail(LBM_ERR_OOM, "host allocation failed");
  gp = &h->g;
  gp->phys = *phys;
  gp->q = phys->lattice == 27 ? 27 : 19;
  gp->phys.lattice = gp->q;
  if (alloc) {
    gp->alloc = *alloc;
    gp->have_alloc = true;
  }
  gp->stream = (cudaStream_t)stream;
  cudaGetDevice(&gp->device);
  *out = h;
  return LBM_OK;
}

// Dense grouping (classification + mapping) from the level's host flags.
static lbm_status dense_groups(Grid& g, Level& L, const float* bc_values, const float* def_bc) {
  const int64_t N = L.n_slots;
  const auto& fl = L.flags_h;
  std::vector<int32_t> regs;
  bool has_wall_voxel = false;
  int64_t n_upd = 0;
  for (int64_t v = 0; v < N; ++v) {
    const int t = flag_type(fl[v]);
    if (type_regularized(t)) regs.push_back((int32_t)v);
    if (type_wall(t)) has_wall_voxel = true;
    if (type_updated(t)) ++n_upd;
    if (!type_updated(t) && !type_wall(t)) return fail(LBM_ERR_INVALID, "unknown voxel type");
  }
  for (int32_t v : regs) {
    if (flag_normal(fl[v]) > 5) return fail(LBM_ERR_INVALID, "regularized voxel with bad normal");
  }
  if (!regs.empty() && !bc_values && !def_bc)
    return fail(LBM_ERR_INVALID, "regularized voxels need bc_values or default_bc");
  L.n_updated = n_upd;
  L.n_reg = (int64_t)regs.size();
  L.dense_reg_tail = !regs.empty() && regs.front() == N - (int64_t)regs.size();
  L.dense_has_flags = has_wall_voxel || !regs.empty();
  // free old tables
  g.dfree(L.flags_d, g.stream);
  g.dfree(L.wmask_d, g.stream);
  g.dfree(L.reg_list_d, g.stream);
  g.dfree(L.bc_grp_d, g.stream);
  g.dfree(L.bc_full_d, g.stream);
  L.flags_d = nullptr;
  L.wmask_d = nullptr;
  L.reg_list_d = nullptr;
  L.bc_grp_d = nullptr;
  L.bc_full_d = nullptr;
  lbm_status st;
  if (L.dense_has_flags) {
    if ((st = upload(g, &L.flags_d, fl.data(), (size_t)N))) return st;
  }
  // per-voxel wall mask when walls are not only the box sides, or when the
  // boundary group is not the contiguous tail
  if (has_wall_voxel || (!regs.empty() && !L.dense_reg_tail)) {
    std::vector<uint32_t> wm;
    if (g.q == 27) q27::dense_wall_mask(g, L, wm);
    else q19::dense_wall_mask(g, L, wm);
    if ((st = upload(g, &L.wmask_d, wm.data(), wm.size()))) return st;
  }
  if (!regs.empty()) {
    if (!L.dense_reg_tail) {
      if ((st = upload(g, &L.reg_list_d, regs.data(), regs.size()))) return st;
    }
    L.bc_h.assign(regs.size() * 4, 0.f);
    for (size_t k = 0; k < regs.size(); ++k)
      for (int c = 0; c < 4; ++c) L.bc_h[k * 4 + c] = bc_values ? bc_values[k * 4 + c] : def_bc[c];
    if ((st = upload(g, &L.bc_grp_d, (const float4*)L.bc_h.data(), regs.size()))) return st;
  }
  return LBM_OK;
}

// Monolithic kernels read boundary values from a full-domain array (the
// naive storage of Table 2); built on first use.
static lbm_status ensure_bc_full(Grid& g, Level& L) {
  if (L.bc_full_d || L.n_reg == 0) return LBM_OK;
  std::vector<float4> full((size_t)L.n_slots, make_float4(0.f, 0.f, 0.f, 1.f));
  if (L.E == 0) {
    size_t k = 0;
    for (int64_t v = 0; v < L.n_slots; ++v)
      if (type_regularized(flag_type(L.flags_h[v]))) {
        full[(size_t)v] = make_float4(L.bc_h[k * 4], L.bc_h[k * 4 + 1], L.bc_h[k * 4 + 2], L.bc_h[k * 4 + 3]);
        ++k;
      }
  } else {
    sparse_fill_bc_full(L, full.data());
  }
  return upload(g, &L.bc_full_d, full.data(), full.size());
}

}  // namespace lbm

using namespace lbm;

extern "C" {

const char* lbm_last_error(void) { return g_last_error.c_str(); }

lbm_status lbm_grid_create_dense(const int dims[3], const lbm_physics* phys,
                                 const lbm_allocator* alloc, void* stream, lbm_grid** out) {
  set_error("");
  if (!dims || dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0)
    return fail(LBM_ERR_INVALID, "dims must be positive");
  if ((double)dims[0] * dims[1] * dims[2] * 27 >= 9.0e18)
    return fail(LBM_ERR_INVALID, "grid too large");
  if (phys && phys->closure) return fail(LBM_ERR_UNSUPPORTED, "the closure runs on multi-resolution grids");
  if (phys && phys->schedule == LBM_SCHEDULE_BITMASK)
    return fail(LBM_ERR_UNSUPPORTED, "bitmask grouping is a block-sparse layout");
  Grid* gp = nullptr;
  lbm_status st = begin(out, phys, alloc, stream, gp);
  if (st) return st;
  Grid& g = *gp;
  g.kind = 0;
  Level& L = g.lv[0];
  L.nx = dims[0];
  L.ny = dims[1];
  L.nz = dims[2];
  L.n_slots = (int64_t)dims[0] * dims[1] * dims[2];
  L.n_updated = L.n_slots;
  L.flags_h.assign((size_t)L.n_slots, 0);
  if ((st = alloc_common(g)) || (st = alloc_populations(g, L))) {
    free_grid(g);
    delete *out;
    *out = nullptr;
    return st;
  }
  return LBM_OK;
}

lbm_status lbm_grid_create_sparse(const int dims[3], int block_edge, const uint8_t* flags,
                                  const lbm_physics* phys, const lbm_allocator* alloc,
                                  void* stream, lbm_grid** out) {
  set_error("");
  if (!dims || dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0)
    return fail(LBM_ERR_INVALID, "dims must be positive");
  if (block_edge != 4 && block_edge != 8) return fail(LBM_ERR_INVALID, "block_edge must be 4 or 8");
  if (!flags) return fail(LBM_ERR_INVALID, "sparse grids need flags");
  for (int a = 0; a < 3; ++a)
    if (phys && phys->periodic[a] && dims[a] % block_edge)
      return fail(LBM_ERR_INVALID, "periodic axes need dims divisible by block_edge");
  if (phys && phys->closure) return fail(LBM_ERR_UNSUPPORTED, "the closure runs on multi-resolution grids");
  Grid* gp = nullptr;
  lbm_status st = begin(out, phys, alloc, stream, gp);
  if (st) return st;
  Grid& g = *gp;
  g.kind = 1;
  Level& L = g.lv[0];
  L.nx = dims[0];
  L.ny = dims[1];
  L.nz = dims[2];
  L.E = block_edge;
  L.flags_h.assign(flags, flags + (size_t)dims[0] * dims[1] * dims[2]);
  if ((st = (g.q == 27 ? q27::sparse_build(g, L) : q19::sparse_build(g, L))) ||
      (st = alloc_common(g)) || (st = alloc_populations(g, L)) ||
      (st = sparse_upload(g, L))) {
    free_grid(g);
    delete *out;
    *out = nullptr;
    return st;
  }
  return LBM_OK;
}

lbm_status lbm_grid_create_multires(const int finest_dims[3], int n_levels,
                                    const uint8_t* level_map, const lbm_physics* phys,
                                    const lbm_allocator* alloc, void* stream, lbm_grid** out) {
  set_error("");
  if (!finest_dims || !level_map) return fail(LBM_ERR_INVALID, "NULL argument");
  if (phys && phys->schedule == LBM_SCHEDULE_BITMASK)
    return fail(LBM_ERR_UNSUPPORTED, "bitmask grouping is a block-sparse layout");
  Grid* gp = nullptr;
  lbm_status st = begin(out, phys, alloc, stream, gp);
  if (st) return st;
  Grid& g = *gp;
  g.kind = 2;
  auto bail = [&](lbm_status s) {
    free_grid(g);
    delete *out;
    *out = nullptr;
    return s;
  };
  if ((st = g.q == 27 ? q27::multires_build(g, finest_dims, n_levels, level_map)
                      : q19::multires_build(g, finest_dims, n_levels, level_map)))
    return bail(st);
  if ((st = alloc_common(g))) return bail(st);
  for (int l = 0; l < g.n_levels; ++l) {
    Level& L = g.lv[l];
    if ((st = alloc_populations(g, L))) return bail(st);
    std::vector<uint8_t> zeros((size_t)std::max<int64_t>(L.n_slots, L.n_blocks), 0);
    if ((st = upload(g, &L.flags_d, zeros.data(), (size_t)L.n_slots)) ||
        (st = upload(g, &L.blk_walls_d, zeros.data(), (size_t)L.n_blocks)) ||
        (st = upload(g, &L.nbr_d, L.nbr_h.data(), L.nbr_h.size())) ||
        (st = upload(g, &L.bmap_d, L.bmap_h.data(), L.bmap_h.size())) ||
        (st = upload(g, &L.coords_d, L.coords_h.data(), L.coords_h.size())) ||
        (st = upload(g, &L.jump_d, L.jump_h.data(), L.jump_h.size())))
      return bail(st);
    L.flags_h.assign((size_t)L.nx * L.ny * L.nz, 0);
    // voxels of regions owned by other levels are "not in domain" on this level
    for (int64_t vb = 0; vb < (int64_t)L.bmap_h.size(); ++vb) {
      if (L.bmap_h[(size_t)vb] >= 0) continue;
      const int bx = (int)(vb % L.nbx), by = (int)((vb / L.nbx) % L.nby),
                bz = (int)(vb / ((int64_t)L.nbx * L.nby));
      for (int l3 = 0; l3 < 512; ++l3) {
        const int x = bx * 8 + (l3 & 7), y = by * 8 + ((l3 >> 3) & 7), z = bz * 8 + (l3 >> 6);
        L.flags_h[x + (size_t)L.nx * (y + (size_t)L.ny * z)] = (uint8_t)T_OUTSIDE;
      }
    }
  }
  if ((st = g.q == 27 ? q27::multires_finish(g) : q19::multires_finish(g))) return bail(st);
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  return LBM_OK;
}

lbm_status lbm_grid_destroy(lbm_grid* h) {
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  free_grid(h->g);
  delete h;
  return LBM_OK;
}

lbm_status lbm_get_info(const lbm_grid* h, lbm_info* out) {
  if (!h || !out) return fail(LBM_ERR_INVALID, "NULL argument");
  const Grid& g = h->g;
  std::memset(out, 0, sizeof(*out));
  out->kind = g.kind;
  out->n_levels = g.n_levels;
  out->dims[0] = g.lv[0].nx;
  out->dims[1] = g.lv[0].ny;
  out->dims[2] = g.lv[0].nz;
  out->block_edge = g.lv[0].E;
  for (int l = 0; l < g.n_levels; ++l) {
    out->n_updated[l] = g.lv[l].n_updated;
    out->n_blocks[l] = g.lv[l].n_blocks;
    out->n_group_b[l] = g.lv[l].n_b;
    out->n_regularized += g.lv[l].n_reg;
    out->population_bytes[l] = g.lv[l].pop_bytes;
  }
  out->steps_done = g.steps_done;
  out->lattice = g.q;
  return LBM_OK;
}

lbm_status lbm_set_schedule(lbm_grid* h, int schedule) {
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  if (schedule != LBM_SCHEDULE_DISAGGREGATED && schedule != LBM_SCHEDULE_MONOLITHIC &&
      schedule != LBM_SCHEDULE_BITMASK)
    return fail(LBM_ERR_INVALID, "unknown schedule");
  // the block order is fixed at creation: a bitmask-grouped grid has no
  // contiguous boundary group, a memory-grouped one no boundary bits
  const bool bm = h->g.kind == 1 && h->g.lv[0].bitmask;
  if ((schedule == LBM_SCHEDULE_BITMASK && !bm) || (schedule == LBM_SCHEDULE_DISAGGREGATED && bm))
    return fail(LBM_ERR_UNSUPPORTED, "the grouping (block order) is chosen at grid creation");
  h->g.phys.schedule = schedule;
  return LBM_OK;
}

lbm_status lbm_set_variant(lbm_grid* h, int variant) {
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  if (variant < 0 || variant > VARIANT_STAGED) return fail(LBM_ERR_INVALID, "unknown variant");
  if (variant == VARIANT_STAGED && (h->g.kind == 0 || h->g.lv[0].E != 8))
    return fail(LBM_ERR_UNSUPPORTED, "the staged variant is a kernel of 8^3-block grids");
  for (int l = 0; l < 4; ++l) h->g.lv[l].variant = variant;
  return LBM_OK;
}

lbm_status lbm_set_wait_limit(lbm_grid* h, int64_t ns) {
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  h->g.staged_wait_ns = ns < 0 ? Grid::kStagedWaitNs : (uint64_t)ns;
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_grid* h, int n_steps, int* chosen, double* ms_per_step) {
  if (!h || n_steps <= 0) return fail(LBM_ERR_INVALID, "bad autotune arguments");
  Grid& g = h->g;
  cudaStream_t s = g.stream;
  // save the state of every level
  std::vector<Scratch*> saved;
  int cur[4];
  for (int l = 0; l < g.n_levels; ++l) {
    Level& L = g.lv[l];
    cur[l] = L.cur;
    saved.push_back(new Scratch(g, L.pop_bytes, s));
    if (!saved.back()->p) {
      for (auto* p : saved) delete p;
      return fail(LBM_ERR_OOM, "autotune scratch allocation failed");
    }
    LBM_CUDA(cudaMemcpyAsync(saved.back()->p, L.f[L.cur], L.pop_bytes, cudaMemcpyDeviceToDevice, s));
  }
  const int64_t steps0 = g.steps_done;
  const int old_variant = g.lv[0].variant;
  double best = 1e30;
  int best_v = old_variant;
  cudaEvent_t e0, e1;
  LBM_CUDA(cudaEventCreate(&e0));
  LBM_CUDA(cudaEventCreate(&e1));
  lbm_status st = LBM_OK;
  // candidates: the dense interior variants, or the block-sparse lean kernel
  // and its staged form (8^3 blocks); the others keep the default kernel
  std::vector<int> cand;
  if (g.kind == 0) {
    for (int v = 0; v < N_VARIANTS; ++v) cand.push_back(v);
  } else {
    cand.push_back(VARIANT_SCALAR);
    if (g.lv[0].E == 8) cand.push_back(VARIANT_STAGED);
  }
  if (ms_per_step)
    for (int v = 0; v <= VARIANT_STAGED; ++v) ms_per_step[v] = 0.0;
  for (size_t c = 0; c < cand.size() && st == LBM_OK; ++c) {
    const int v = cand[c];
    for (int l = 0; l < g.n_levels; ++l) g.lv[l].variant = v;
    st = lbm_step(h, 2, s);  // warm-up of this variant
    if (st) break;
    cudaEventRecord(e0, s);
    st = lbm_step(h, n_steps, s);
    cudaEventRecord(e1, s);
    if (st) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / n_steps;
    if (ms_per_step) ms_per_step[v] = per;
    if (per < best) {
      best = per;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int l = 0; l < g.n_levels; ++l) {
    Level& L = g.lv[l];
    L.cur = cur[l];
    cudaMemcpyAsync(L.f[L.cur], saved[(size_t)l]->p, L.pop_bytes, cudaMemcpyDeviceToDevice, s);
    L.variant = st == LBM_OK ? best_v : old_variant;
  }
  cudaStreamSynchronize(s);
  for (auto* p : saved) delete p;
  g.steps_done = steps0;
  if (st) return st;
  if (chosen) *chosen = best_v;
  return LBM_OK;
}

lbm_status lbm_set_boundary(lbm_grid* h, int level, const uint8_t* flags,
                            const float* bc_values, const float default_bc[4]) {
  set_error("");
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  Grid& g = h->g;
  if (level < 0 || level >= g.n_levels) return fail(LBM_ERR_INVALID, "bad level");
  Level& L = g.lv[level];
  const size_t nv = (size_t)L.nx * L.ny * L.nz;
  if (g.kind == 0) {
    std::vector<uint8_t> keep = L.flags_h;
    if (flags) L.flags_h.assign(flags, flags + nv);
    lbm_status st = dense_groups(g, L, bc_values, default_bc);
    if (st) {
      L.flags_h.swap(keep);
      dense_groups(g, L, nullptr, nullptr);
      return st;
    }
    return LBM_OK;
  }
  if (g.kind == 2 && level == 0)
    return g.q == 27 ? q27::multires_set_boundary(g, flags, bc_values, default_bc)
                     : q19::multires_set_boundary(g, flags, bc_values, default_bc);
  if (flags && std::memcmp(flags, L.flags_h.data(), nv) != 0)
    return fail(LBM_ERR_INVALID, "sparse flags (and those of multi-resolution levels >= 1) are fixed at creation");
  return sparse_set_bc(g, L, bc_values, default_bc);
}

lbm_status lbm_init_equilibrium(lbm_grid* h, int level, const double* rho, const double* u,
                                int device_ptrs) {
  set_error("");
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  Grid& g = h->g;
  if (level < 0 || level >= g.n_levels) return fail(LBM_ERR_INVALID, "bad level");
  Level& L = g.lv[level];
  const size_t n = (size_t)L.nx * L.ny * L.nz;
  cudaStream_t s = g.stream;
  if (device_ptrs) {
    lbm_status st = g.q == 27 ? q27::launch_init_equilibrium(g, L, rho, u, s)
                              : q19::launch_init_equilibrium(g, L, rho, u, s);
    if (st) return st;
    LBM_CUDA(cudaStreamSynchronize(s));
    return LBM_OK;
  }
  // page-locked host arrays mapped into the device address space are read
  // by the kernel in place (one pass over the host link, no staging copy)
  const double* mr = mapped_host(rho);
  const double* mu = mapped_host(u);
  if ((!rho || mr) && (!u || mu)) {
    lbm_status st = g.q == 27 ? q27::launch_init_equilibrium(g, L, mr, mu, s)
                              : q19::launch_init_equilibrium(g, L, mr, mu, s);
    if (st) return st;
    LBM_CUDA(cudaStreamSynchronize(s));
    return LBM_OK;
  }
  Scratch dr(g, rho ? n * sizeof(double) : 16, s), du(g, u ? 3 * n * sizeof(double) : 16, s);
  if (!dr.p || !du.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  if (rho) LBM_CUDA(cudaMemcpyAsync(dr.p, rho, n * sizeof(double), cudaMemcpyHostToDevice, s));
  if (u) LBM_CUDA(cudaMemcpyAsync(du.p, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
  const double* rp = rho ? (const double*)dr.p : nullptr;
  const double* up = u ? (const double*)du.p : nullptr;
  lbm_status st = g.q == 27 ? q27::launch_init_equilibrium(g, L, rp, up, s)
                            : q19::launch_init_equilibrium(g, L, rp, up, s);
  if (st) return st;
  LBM_CUDA(cudaStreamSynchronize(s));
  return LBM_OK;
}

lbm_status lbm_step(lbm_grid* h, int n_steps, void* stream) {
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  if (n_steps < 0) return fail(LBM_ERR_INVALID, "n_steps < 0");
  Grid& g = h->g;
  for (int l = 0; l < g.n_levels; ++l)
    if (g.lv[l].n_reg > 0 && g.lv[l].bc_h.size() != (size_t)g.lv[l].n_reg * 4)
      return fail(LBM_ERR_INVALID, "regularized voxels have no boundary values (lbm_set_boundary)");
  cudaStream_t s = stream ? (cudaStream_t)stream : g.stream;
  if (s != g.stream) {
    if (!g.stream_ev) LBM_CUDA(cudaEventCreateWithFlags(&g.stream_ev, cudaEventDisableTiming));
    LBM_CUDA(cudaEventRecord(g.stream_ev, g.stream));
    LBM_CUDA(cudaStreamWaitEvent(s, g.stream_ev, 0));
  }
  g.stream = s;
  if (g.phys.schedule == LBM_SCHEDULE_MONOLITHIC) {
    for (int l = 0; l < g.n_levels; ++l) {
      lbm_status st = ensure_bc_full(g, g.lv[l]);
      if (st) return st;
    }
  }
  for (int k = 0; k < n_steps; ++k) {
    lbm_status st = g.kind == 0   ? (g.q == 27 ? q27::dense_step(g, g.lv[0], s)
                                               : q19::dense_step(g, g.lv[0], s))
                    : g.kind == 1 ? (g.q == 27 ? q27::sparse_step(g, g.lv[0], s)
                                               : q19::sparse_step(g, g.lv[0], s))
                                  : (g.q == 27 ? q27::multires_step(g, s, k == 0) : q19::multires_step(g, s, k == 0));
    if (st) return st;
    ++g.steps_done;
  }
  return LBM_OK;
}

lbm_status lbm_sync(lbm_grid* h) {
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  Grid& g = h->g;
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  int st = 0;
  LBM_CUDA(cudaMemcpy(&st, g.status_d, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    LBM_CUDA(cudaMemset(g.status_d, 0, sizeof(int)));
    return fail((lbm_status)st, "device status latched");
  }
  return LBM_OK;
}

lbm_status lbm_get_moments(lbm_grid* h, int level, double* rho, double* u, int device_ptrs) {
  set_error("");
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  Grid& g = h->g;
  if (level < 0 || level >= g.n_levels) return fail(LBM_ERR_INVALID, "bad level");
  lbm_status st = lbm_sync(h);
  if (st) return st;
  Level& L = g.lv[level];
  const size_t n = (size_t)L.nx * L.ny * L.nz;
  cudaStream_t s = g.stream;
  if (device_ptrs) {
    if ((st = g.q == 27 ? q27::launch_moments(g, L, rho, u, s)
                        : q19::launch_moments(g, L, rho, u, s)))
      return st;
    LBM_CUDA(cudaStreamSynchronize(s));
    return LBM_OK;
  }
  // page-locked host arrays mapped into the device address space are written
  // by the kernel in place
  double* mr = mapped_host(rho);
  double* mu = mapped_host(u);
  if ((!rho || mr) && (!u || mu)) {
    if ((st = g.q == 27 ? q27::launch_moments(g, L, mr, mu, s) : q19::launch_moments(g, L, mr, mu, s)))
      return st;
    LBM_CUDA(cudaStreamSynchronize(s));
    return LBM_OK;
  }
  Scratch dr(g, rho ? n * sizeof(double) : 16, s), du(g, u ? 3 * n * sizeof(double) : 16, s);
  if (!dr.p || !du.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  double* rp = rho ? (double*)dr.p : nullptr;
  double* up = u ? (double*)du.p : nullptr;
  if ((st = g.q == 27 ? q27::launch_moments(g, L, rp, up, s) : q19::launch_moments(g, L, rp, up, s)))
    return st;
  if (rho) LBM_CUDA(cudaMemcpyAsync(rho, dr.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (u) LBM_CUDA(cudaMemcpyAsync(u, du.p, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_grid* h, int level, void* dst, size_t bytes, int device_ptrs) {
  if (!h || !dst) return fail(LBM_ERR_INVALID, "NULL argument");
  Grid& g = h->g;
  if (level < 0 || level >= g.n_levels) return fail(LBM_ERR_INVALID, "bad level");
  Level& L = g.lv[level];
  if (bytes != L.pop_bytes) return fail(LBM_ERR_INVALID, "bytes != population_bytes");
  lbm_status st = lbm_sync(h);
  if (st) return st;
  LBM_CUDA(cudaMemcpyAsync(dst, L.f[L.cur], bytes,
                           device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g.stream));
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_grid* h, int level, const void* src, size_t bytes,
                               int device_ptrs) {
  if (!h || !src) return fail(LBM_ERR_INVALID, "NULL argument");
  Grid& g = h->g;
  if (level < 0 || level >= g.n_levels) return fail(LBM_ERR_INVALID, "bad level");
  Level& L = g.lv[level];
  if (bytes != L.pop_bytes) return fail(LBM_ERR_INVALID, "bytes != population_bytes");
  LBM_CUDA(cudaMemcpyAsync(L.f[L.cur], src, bytes,
                           device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g.stream));
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  return LBM_OK;
}

lbm_status lbm_get_populations_f64(lbm_grid* h, int level, double* dst, int device_ptrs) {
  if (!h || !dst) return fail(LBM_ERR_INVALID, "NULL argument");
  Grid& g = h->g;
  if (level < 0 || level >= g.n_levels) return fail(LBM_ERR_INVALID, "bad level");
  lbm_status st = lbm_sync(h);
  if (st) return st;
  Level& L = g.lv[level];
  const size_t n = (size_t)L.nx * L.ny * L.nz * g.q;
  cudaStream_t s = g.stream;
  if (device_ptrs) {
    if ((st = g.q == 27 ? q27::launch_decode_f64(g, L, dst, s) : q19::launch_decode_f64(g, L, dst, s)))
      return st;
    LBM_CUDA(cudaStreamSynchronize(s));
    return LBM_OK;
  }
  Scratch d(g, n * sizeof(double), s);
  if (!d.p) return fail(LBM_ERR_OOM, "scratch allocation failed");
  if ((st = g.q == 27 ? q27::launch_decode_f64(g, L, (double*)d.p, s)
                      : q19::launch_decode_f64(g, L, (double*)d.p, s)))
    return st;
  LBM_CUDA(cudaMemcpyAsync(dst, d.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  return LBM_OK;
}

lbm_status lbm_layout_bytes(const lbm_grid* h, int level, int what, size_t* bytes) {
  if (!h || !bytes) return fail(LBM_ERR_INVALID, "NULL argument");
  const Grid& g = h->g;
  if (level < 0 || level >= g.n_levels) return fail(LBM_ERR_INVALID, "bad level");
  const Level& L = g.lv[level];
  switch (what) {
    case LBM_LAYOUT_FLAGS: *bytes = L.flags_h.size(); return LBM_OK;
    case LBM_LAYOUT_BLOCK_COORDS: *bytes = L.coords_h.size() * 4; return LBM_OK;
    case LBM_LAYOUT_NBR: *bytes = L.nbr_h.size() * 4; return LBM_OK;
    case LBM_LAYOUT_BLOCK_MAP: *bytes = L.bmap_h.size() * 4; return LBM_OK;
    case LBM_LAYOUT_XNBR_COARSE:
      if (g.kind != 2) break;
      *bytes = L.xnbr_coarse_h.size() * 4;
      return LBM_OK;
    case LBM_LAYOUT_XNBR_FINE:
      if (g.kind != 2) break;
      *bytes = L.xnbr_fine_h.size() * 4;
      return LBM_OK;
    case LBM_LAYOUT_BOUNDARY_BITS:
      if (!L.bitmask) break;
      *bytes = L.bnd_bits_h.size() * 4;
      return LBM_OK;
    case LBM_LAYOUT_BC_INDEX:
      if (!L.bitmask) break;
      *bytes = L.bc_idx_h.size() * 4;
      return LBM_OK;
    case LBM_LAYOUT_IFACE_SLOTS:
    case LBM_LAYOUT_IFACE_CROSS:
      if (g.kind != 2) break;
      *bytes = (size_t)L.n_iface * 4;
      return LBM_OK;
    default: break;
  }
  return fail(LBM_ERR_UNSUPPORTED, "layout table not available for this grid");
}

lbm_status lbm_get_layout(const lbm_grid* h, int level, int what, void* dst, size_t bytes) {
  size_t need = 0;
  lbm_status st = lbm_layout_bytes(h, level, what, &need);
  if (st) return st;
  if (!dst || bytes != need) return fail(LBM_ERR_INVALID, "bytes != layout table size");
  const Level& L = h->g.lv[level];
  const void* src = what == LBM_LAYOUT_FLAGS ? (const void*)L.flags_h.data()
                    : what == LBM_LAYOUT_BLOCK_COORDS ? (const void*)L.coords_h.data()
                    : what == LBM_LAYOUT_NBR ? (const void*)L.nbr_h.data()
                    : what == LBM_LAYOUT_BLOCK_MAP ? (const void*)L.bmap_h.data()
                    : what == LBM_LAYOUT_XNBR_COARSE ? (const void*)L.xnbr_coarse_h.data()
                    : what == LBM_LAYOUT_XNBR_FINE ? (const void*)L.xnbr_fine_h.data()
                    : what == LBM_LAYOUT_BOUNDARY_BITS ? (const void*)L.bnd_bits_h.data()
                    : what == LBM_LAYOUT_IFACE_SLOTS ? (const void*)L.iface_slot_h.data()
                    : what == LBM_LAYOUT_IFACE_CROSS ? (const void*)L.iface_cross_h.data()
                                                       : (const void*)L.bc_idx_h.data();
  if (need) std::memcpy(dst, src, need);
  return LBM_OK;
}

lbm_status lbm_profile(lbm_grid* h, int enable) {
  if (!h) return fail(LBM_ERR_INVALID, "grid is NULL");
  Grid& g = h->g;
  if (enable) {
    LBM_CUDA(cudaStreamSynchronize(g.stream));
    prof_clear(g);
  }
  g.prof = enable != 0;
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_grid* h, lbm_kernel_stat* out, int max, int* n_out) {
  if (!h || !n_out || (max > 0 && !out)) return fail(LBM_ERR_INVALID, "NULL argument");
  Grid& g = h->g;
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  const int nk = (int)g.prof_names.size();
  *n_out = nk;
  for (int k = 0; k < nk && k < max; ++k) {
    std::memset(&out[k], 0, sizeof(out[k]));
    std::strncpy(out[k].name, g.prof_names[(size_t)k].c_str(), sizeof(out[k].name) - 1);
  }
  for (const auto& r : g.prof_recs) {
    if (r.kernel >= max) continue;
    float ms = 0.f;
    LBM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    out[r.kernel].launches += 1;
    out[r.kernel].total_ms += ms;
    out[r.kernel].units += r.units;
  }
  return LBM_OK;
}

lbm_status lbm_profile_trace(lbm_grid* h, lbm_kernel_trace* out, int max, int* n_out) {
  if (!h || !n_out || (max > 0 && !out)) return fail(LBM_ERR_INVALID, "NULL argument");
  Grid& g = h->g;
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  const int n = (int)g.prof_recs.size();
  *n_out = n;
  if (n == 0) return LBM_OK;
  const cudaEvent_t t0 = g.prof_recs[0].a;
  for (int k = 0; k < n && k < max; ++k) {
    const ProfRec& r = g.prof_recs[(size_t)k];
    std::memset(&out[k], 0, sizeof(out[k]));
    std::strncpy(out[k].name, g.prof_names[(size_t)r.kernel].c_str(), sizeof(out[k].name) - 1);
    float a = 0.f, b = 0.f;
    LBM_CUDA(cudaEventElapsedTime(&a, t0, r.a));
    LBM_CUDA(cudaEventElapsedTime(&b, t0, r.b));
    out[k].start_ms = a;
    out[k].end_ms = b;
    out[k].units = r.units;
  }
  return LBM_OK;
}

lbm_status lbm_conservation(lbm_grid* h, double out[4]) {
  if (!h || !out) return fail(LBM_ERR_INVALID, "NULL argument");
  Grid& g = h->g;
  lbm_status st = lbm_sync(h);
  if (st) return st;
  if ((st = g.q == 27 ? q27::launch_conservation(g, g.sums_d, g.stream)
                      : q19::launch_conservation(g, g.sums_d, g.stream)))
    return st;
  LBM_CUDA(cudaMemcpyAsync(out, g.sums_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, g.stream));
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(out[k])) return fail(LBM_ERR_DIVERGED, "non-finite mass or momentum");
  return LBM_OK;
}

}  // extern "C"
