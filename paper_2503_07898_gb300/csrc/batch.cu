// batch.cu - many independent simulations in one persistent launch per step.
//
// Not in the paper (a serving-style use of the same update): a batch holds
// dense and 8^3 block-sparse grids of different sizes, walls and relaxation
// times.  Their voxels are cut into work items of 512 voxels (dense: 512
// consecutive voxel ids; sparse: one 8^3 block), two per thread, listed case
// after case; one
// persistent kernel per step walks the list with a grid-stride loop, so a
// step over the whole batch is a single launch whatever the number of cases.
// A sequence of steps is captured once into a CUDA graph and replayed.  The
// persistent grid size (CTAs per SM) is the tuning knob of lbm_batch_autotune.
// Cases running the learned closure are listed after all the others and
// stepped by a second persistent launch of the closure kernel variant, so
// its larger register and shared-memory footprint costs the other cases
// nothing.
#include <algorithm>
#include <map>
#include <vector>

#include "closure.cuh"
#include "d3q19.cuh"
#include "dense.cuh"
#include "grid.h"
#include "sparse.cuh"

namespace lbm {

struct BatchCase {
  int kind;  // 0 dense, 1 sparse (block edge 8)
  int nx, ny, nz, px, py, pz;
  int64_t N;                 // dense voxels / sparse slots
  const uint32_t* wmask;     // per-voxel (dense) or per-slot (sparse) wall mask; dense: null
                             // when walls are only at box sides
  const uint8_t* flags;      // sparse slot flags
  const int32_t* nbr;        // sparse neighbour table
  const uint8_t* blk_walls;  // sparse per-block wall bit
  void* buf[2];
  int cur0;  // buffer holding the state before step parity 0
  float omega;
  float tau;
  int closure;  // learned closure on this case (lbm_batch_closure_load)
  float inv_nx, inv_ny;  // dense: 1 / nx, 1 / ny (voxel decode)
};

constexpr int BT = 256;       // threads per CTA
constexpr int VPT = 2;        // voxels per thread in a work item, taken one after the other
constexpr int VPI = BT * VPT; // voxels per work item: 512 (dense: consecutive ids; sparse: a block)

template <int S, int COLL, bool CLOSURE>
__global__ void __launch_bounds__(BT, (S == S_F32 || CLOSURE) ? 1 : 5) batch_step_kernel(const BatchCase* __restrict__ cases,
                                                        const int32_t* __restrict__ item_case,
                                                        const int32_t* __restrict__ item_local,
                                                        int64_t n_items, int parity,
                                                        const ClosureParams* __restrict__ cp) {
  using T = typename Codec<S>::T;
  extern __shared__ __align__(16) unsigned char batch_dyn_smem[];
  if constexpr (CLOSURE) {
    closure_load_smem(reinterpret_cast<ClosureCta*>(batch_dyn_smem)->w, cp);
    __syncthreads();
  }
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const BatchCase& C = cases[item_case[it]];
    const int64_t t = item_local[it];
    const int in = parity ^ C.cur0;
    const T* __restrict__ fin = (const T*)C.buf[in];
    T* __restrict__ fout = (T*)C.buf[in ^ 1];
    // the item's VPT voxels of this thread, one after the other: the item
    // lookup and the case's descriptor serve them all
#pragma unroll 1
    for (int h = 0; h < VPT; ++h) {
      float g[Q];
      bool act;
      bool inb = true;  // a voxel of the case (dense: the last item's tail lies past it)
      int64_t obase;  // output index of population 0; population I adds I * ostride
      int ostride;
      if (C.kind == 0) {
        // case sizes are below 2^31 / 19 voxels (checked at creation): 32-bit
        // voxel ids and offsets
        // the item's first voxel, packed x | y << 11 | z << 22; this thread's
        // voxel follows by carrying across rows and planes with a float
        // reciprocal (exact: x and y stay below 2^12, so the product's error
        // is far below the 0.5 / n distance to the next integer)
        const uint32_t pk = (uint32_t)t;
        int x = (int)(pk & 2047u) + h * BT + (int)threadIdx.x, y = (int)((pk >> 11) & 2047u),
            z = (int)(pk >> 22);
        int k = (int)(((float)x + 0.5f) * C.inv_nx);
        x -= k * C.nx;
        y += k;
        k = (int)(((float)y + 0.5f) * C.inv_ny);
        y -= k * C.ny;
        z += k;
        const int v = x + C.nx * (y + C.ny * z);
        uint32_t wm = 0u;
        act = inb = z < C.nz;
        if (act && C.wmask) {
          wm = C.wmask[v];
          act = !(wm & (WM_SKIP | WM_REG));
        }
        // one pull form per warp: with a wall bit in any lane, the whole warp
        // takes the wall-mask form (a lane without bits selects nothing), so
        // a warp never runs both forms one after the other
        const bool wmw = __any_sync(0xffffffffu, wm != 0u);
        obase = v;
        ostride = (int)C.N;
        if (act) {
          DenseArgs a{};
          a.nx = C.nx;
          a.ny = C.ny;
          a.nz = C.nz;
          a.N = C.N;
          a.px = C.px;
          a.py = C.py;
          a.pz = C.pz;
          if (lean_row(a, y, z)) {
            if (wmw) pull_row_interior<S, int, true>(fin, a, x, y, z, v, wm, g);
            else pull_row_interior<S, int, false>(fin, a, x, y, z, v, 0u, g);
          } else {
            pull_all<S>(fin, a, x, y, z, v, wm, g);
          }
        } else {
  #pragma unroll
          for (int i = 0; i < Q; ++i) g[i] = 0.f;  // rest state (solid voxel)
        }
      } else {
        const int b = (int)t;
        const int l = h * BT + (int)threadIdx.x;
        const bool walls = C.blk_walls[b] != 0;
        uint32_t wm = 0u;
        if (walls) wm = C.wmask[(int64_t)b * 512 + l];
        act = !(wm & WM_SKIP);
        obase = (int64_t)b * (Q * 512) + l;
        ostride = 512;
        if (act) {
          // batch cases hold fewer than 2^31 / 19 slots: 32-bit offsets
          sparse_pull_voxel<S, 8, int32_t>(fin, C.nbr + (int64_t)b * 27, wm, b, l, walls, g);
        } else {
  #pragma unroll
          for (int i = 0; i < Q; ++i) g[i] = 0.f;  // rest state (solid voxel)
        }
      }
      float omega = C.omega;
      float m[4];            // moments of g, formed with the features
      bool have_m = false;
      if constexpr (CLOSURE) {
        if (C.closure) {  // uniform per item: every lane of every warp takes part
          // a lane without a voxel (past the case's end) joins with the rest state
          if (!inb) {
  #pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = 0.f;
          }
          ClosureCta* sm = reinterpret_cast<ClosureCta*>(batch_dyn_smem);
          float x[MLP_IN];
          closure_features(g, C.tau, x, m);
          have_m = true;
          const float dtau = mlp_bf16_warp(x, sm->w, sm->stage[threadIdx.x >> 5]);
          omega = 1.f / fmaxf(C.tau + dtau, TAU_MIN);
        }
      }
      if (inb) {
        // a voxel that is not updated (solid) carries the rest state (g = 0)
        // through the collision, which keeps it, and stores it: batch cases
        // have no other writer, and whole-sector stores spare the DRAM read
        // that completes a partly written sector (ECC memory)
        if (have_m) collide_m<COLL>(g, omega, m[0], m[1], m[2], m[3]);
        else collide<COLL>(g, omega);
        // one base pointer; the population stride is a constant for sparse
        // items (512) and a 32-bit value for dense ones
        T* __restrict__ o = fout + obase;
        if (C.kind == 0) {
          static_for<Q>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            o[I * ostride] = Codec<S>::template store<I>(g[I]);
          });
        } else {
          static_for<Q>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            o[I * 512] = Codec<S>::template store<I>(g[I]);
          });
        }
      }
    }
  }
}

template <int S, int COLL, bool CLOSURE>
static void launch_step(const BatchCase* cases, const int32_t* ic, const int32_t* il,
                        int64_t n_items, int grid, int parity, const ClosureParams* cp,
                        cudaStream_t s) {
  const size_t smem = CLOSURE ? sizeof(ClosureCta) : 0;
  batch_step_kernel<S, COLL, CLOSURE><<<grid, BT, smem, s>>>(cases, ic, il, n_items, parity, cp);
}

using StepFn = void (*)(const BatchCase*, const int32_t*, const int32_t*, int64_t, int, int,
                        const ClosureParams*, cudaStream_t);

template <bool CL>
static StepFn step_fn_t(int storage, int collision) {
  const bool bgk = collision == C_BGK;
  switch (storage) {
    case S_F32: return bgk ? launch_step<S_F32, C_BGK, CL> : launch_step<S_F32, C_REG, CL>;
    case S_F16: return bgk ? launch_step<S_F16, C_BGK, CL> : launch_step<S_F16, C_REG, CL>;
    default: return bgk ? launch_step<S_BF16, C_BGK, CL> : launch_step<S_BF16, C_REG, CL>;
  }
}

static StepFn step_fn(int storage, int collision, bool closure) {
  return closure ? step_fn_t<true>(storage, collision) : step_fn_t<false>(storage, collision);
}

}  // namespace lbm

using namespace lbm;

struct lbm_batch {
  std::vector<lbm_grid*> grids;
  std::vector<BatchCase> cases_h;
  BatchCase* cases_d = nullptr;
  int32_t* item_case_d = nullptr;
  int32_t* item_local_d = nullptr;
  int64_t n_items = 0;
  int64_t n_plain = 0;                        // items of cases without the closure (listed first)
  std::vector<int32_t> items_per_case;
  std::vector<int64_t> item_first;      // per case: its first item in creation order
  std::vector<int32_t> item_local_h;    // per item in creation order: its local code
  int64_t n_updated = 0;
  int storage = 0, collision = 0;
  int n_sm = 1;
  int ctas_per_sm = 4;
  ClosureParams* cp_d = nullptr;              // learned closure weights (device)
  bool closure = false;                       // some case runs the closure
  cudaStream_t cap = nullptr;                 // capture stream (non-blocking)
  std::map<int, cudaGraphExec_t> graphs;      // steps -> instantiated graph
  StepFn fn = nullptr;      // plain kernel
  StepFn fn_cl = nullptr;   // closure kernel (items n_plain .. n_items)

  int grid_size() const { return n_sm * ctas_per_sm; }
  // one step: plain items, then the closure items (if any)
  void launch(int grid, int parity, cudaStream_t s) const {
    if (n_plain > 0) fn(cases_d, item_case_d, item_local_d, n_plain, grid, parity, cp_d, s);
    if (n_items > n_plain)
      fn_cl(cases_d, item_case_d + n_plain, item_local_d + n_plain, n_items - n_plain, grid,
            parity, cp_d, s);
  }
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
};

static void batch_free(lbm_batch* b) {
  if (!b) return;
  b->drop_graphs();
  cudaFree(b->cases_d);
  cudaFree(b->item_case_d);
  cudaFree(b->item_local_d);
  cudaFree(b->cp_d);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

// Re-upload descriptors if a case advanced on its own since the last upload.
static lbm_status sync_descriptors(lbm_batch* b, cudaStream_t s) {
  bool dirty = false;
  for (size_t c = 0; c < b->grids.size(); ++c) {
    const int cur = b->grids[c]->g.lv[0].cur;
    if (b->cases_h[c].cur0 != cur) {
      b->cases_h[c].cur0 = cur;
      dirty = true;
    }
  }
  if (dirty)
    LBM_CUDA(cudaMemcpyAsync(b->cases_d, b->cases_h.data(), b->cases_h.size() * sizeof(BatchCase),
                             cudaMemcpyHostToDevice, s));
  return LBM_OK;
}

static void advance_bookkeeping(lbm_batch* b, int n) {
  for (auto* h : b->grids) {
    Level& L = h->g.lv[0];
    if (n & 1) L.cur ^= 1;
    h->g.steps_done += n;
  }
}

extern "C" {

lbm_status lbm_batch_create(int n_cases, lbm_grid* const* cases, lbm_batch** out) {
  set_error("");
  if (!out || !cases || n_cases <= 0) return fail(LBM_ERR_INVALID, "bad batch arguments");
  *out = nullptr;
  lbm_batch* b = new lbm_batch();
  std::vector<int32_t> ic, il;
  for (int c = 0; c < n_cases; ++c) {
    lbm_grid* h = cases[c];
    if (!h) {
      batch_free(b);
      return fail(LBM_ERR_INVALID, "NULL case");
    }
    const Grid& g = h->g;
    const Level& L = g.lv[0];
    if (c == 0) {
      b->storage = g.phys.storage;
      b->collision = g.phys.collision;
    }
    const char* why = nullptr;
    if (g.kind == 2) why = "multi-resolution grids cannot join a batch";
    else if (g.q != 19) why = "batches are D3Q19";
    else if (g.phys.storage != b->storage || g.phys.collision != b->collision)
      why = "all cases need the same storage and collision";
    else if (L.n_reg > 0) why = "cases with regularized boundaries cannot join a batch";
    else if (g.kind == 1 && L.E != 8) why = "sparse cases need 8^3 blocks";
    else if (L.n_slots * Q >= ((int64_t)1 << 31)) why = "case too large for a batch (19 N >= 2^31)";
    else if (g.kind == 0 && (L.nx > 2047 || L.ny > 2047 || L.nz > 1023))
      why = "dense batch cases need nx, ny <= 2047 and nz <= 1023";
    if (why) {
      batch_free(b);
      return fail(LBM_ERR_UNSUPPORTED, why);
    }
    BatchCase d{};
    d.kind = g.kind;
    d.nx = L.nx;
    d.ny = L.ny;
    d.nz = L.nz;
    d.px = g.phys.periodic[0];
    d.py = g.phys.periodic[1];
    d.pz = g.phys.periodic[2];
    d.N = L.n_slots;
    d.wmask = L.wmask_d;
    d.flags = L.flags_d;
    d.nbr = L.nbr_d;
    d.blk_walls = L.blk_walls_d;
    d.buf[0] = L.f[0];
    d.buf[1] = L.f[1];
    d.cur0 = L.cur;
    d.omega = (float)(1.0 / g.phys.tau);
    d.tau = (float)g.phys.tau;
    d.closure = 0;
    d.inv_nx = 1.f / (float)L.nx;
    d.inv_ny = 1.f / (float)L.ny;
    b->cases_h.push_back(d);
    const int64_t items = g.kind == 0 ? (L.n_slots + VPI - 1) / VPI : L.n_blocks;
    for (int64_t t = 0; t < items; ++t) {
      ic.push_back(c);
      if (g.kind == 0) {  // dense: first voxel of the item, packed
        const int64_t v0 = t * VPI;
        const int64_t x0 = v0 % L.nx, y0 = (v0 / L.nx) % L.ny, z0 = v0 / ((int64_t)L.nx * L.ny);
        il.push_back((int32_t)(uint32_t)(x0 | (y0 << 11) | (z0 << 22)));
      } else {
        il.push_back((int32_t)t);
      }
    }
    b->items_per_case.push_back((int32_t)items);
    b->n_updated += L.n_updated;
    b->grids.push_back(h);
  }
  b->n_items = (int64_t)ic.size();
  b->n_plain = b->n_items;
  b->item_local_h = il;
  {
    int64_t first = 0;
    for (int32_t n : b->items_per_case) {
      b->item_first.push_back(first);
      first += n;
    }
  }
  b->fn = step_fn(b->storage, b->collision, false);
  b->fn_cl = step_fn(b->storage, b->collision, true);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMalloc(&b->cases_d, b->cases_h.size() * sizeof(BatchCase));
  if (e == cudaSuccess) e = cudaMalloc(&b->item_case_d, ic.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&b->item_local_d, il.size() * 4);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->cases_d, b->cases_h.data(), b->cases_h.size() * sizeof(BatchCase),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->item_case_d, ic.data(), ic.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->item_local_d, il.data(), il.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "lbm_batch_create");
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
  cudaDeviceSynchronize();
  batch_free(b);
  return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch* b, int64_t* n_updated, int64_t* n_items,
                          int* ctas_per_sm) {
  if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
  if (n_updated) *n_updated = b->n_updated;
  if (n_items) *n_items = b->n_items;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  return LBM_OK;
}

lbm_status lbm_batch_closure_load(lbm_batch* b, const float* theta, size_t n, int max_edge) {
  set_error("");
  if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
  if (max_edge > 0 && !theta) return fail(LBM_ERR_INVALID, "NULL weights");
  if (max_edge > 0 && n != (size_t)MLP_PARAMS)
    return fail(LBM_ERR_INVALID, "closure weights must have 5313 values");
  cudaStream_t s = b->cap;
  if (max_edge > 0) {
    ClosureParams cp;
    closure_params_from_fp32(theta, &cp);
    if (!b->cp_d) LBM_CUDA(cudaMalloc(&b->cp_d, sizeof(ClosureParams)));
    LBM_CUDA(cudaMemcpyAsync(b->cp_d, &cp, sizeof(cp), cudaMemcpyHostToDevice, s));
  }
  // the work list: items of plain cases first, then those of closure cases
  std::vector<int32_t> ic, il;
  for (int pass = 0; pass < 2; ++pass)
    for (size_t c = 0; c < b->cases_h.size(); ++c) {
      BatchCase& d = b->cases_h[c];
      d.closure = max_edge > 0 && std::max(d.nx, std::max(d.ny, d.nz)) <= max_edge;
      if (d.closure != pass) continue;
      for (int32_t t = 0; t < b->items_per_case[c]; ++t) {
        ic.push_back((int32_t)c);
        il.push_back(b->item_local_h[(size_t)(b->item_first[c] + t)]);
      }
    }
  if (ic.size() != (size_t)b->n_items) return fail(LBM_ERR_INTERNAL, "batch work list size");
  int64_t n_plain = 0;
  while (n_plain < b->n_items && !b->cases_h[(size_t)ic[(size_t)n_plain]].closure) ++n_plain;
  LBM_CUDA(cudaMemcpyAsync(b->cases_d, b->cases_h.data(), b->cases_h.size() * sizeof(BatchCase),
                           cudaMemcpyHostToDevice, s));
  LBM_CUDA(cudaMemcpyAsync(b->item_case_d, ic.data(), ic.size() * 4, cudaMemcpyHostToDevice, s));
  LBM_CUDA(cudaMemcpyAsync(b->item_local_d, il.data(), il.size() * 4, cudaMemcpyHostToDevice, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  b->n_plain = n_plain;
  b->closure = n_plain < b->n_items;
  b->drop_graphs();
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n_steps, void* stream) {
  if (!b || n_steps < 0) return fail(LBM_ERR_INVALID, "bad batch_step arguments");
  if (n_steps == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  lbm_status st = sync_descriptors(b, s);
  if (st) return st;
  auto it = b->graphs.find(n_steps);
  if (it == b->graphs.end()) {
    // capture n_steps persistent launches once; parity k & 1 per step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    LBM_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < n_steps; ++k)
      b->launch(b->grid_size(), k & 1, b->cap);
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
    it = b->graphs.emplace(n_steps, exec).first;
  }
  LBM_CUDA(cudaGraphLaunch(it->second, s));
  advance_bookkeeping(b, n_steps);
  return sync_descriptors(b, s);
}

lbm_status lbm_batch_autotune(lbm_batch* b, int n_steps, int* chosen, double* ms_per_step) {
  if (!b || n_steps <= 0) return fail(LBM_ERR_INVALID, "bad batch_autotune arguments");
  const int cand[6] = {1, 2, 3, 4, 6, 8};
  cudaStream_t s = b->cap;
  lbm_status st = sync_descriptors(b, s);
  if (st) return st;
  // save every case's state
  size_t total = 0;
  for (auto* h : b->grids) total += h->g.lv[0].pop_bytes;
  void* save = nullptr;
  LBM_CUDA(cudaMalloc(&save, total));
  size_t off = 0;
  for (auto* h : b->grids) {
    const Level& L = h->g.lv[0];
    cudaMemcpyAsync((char*)save + off, L.f[L.cur], L.pop_bytes, cudaMemcpyDeviceToDevice, s);
    off += L.pop_bytes;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  int best_k = b->ctas_per_sm;
  for (int c = 0; c < 6; ++c) {
    const int grid = b->n_sm * cand[c];
    b->launch(grid, 0, s);  // warm-up
    b->launch(grid, 1, s);
    cudaEventRecord(e0, s);
    for (int k = 0; k < n_steps; ++k)
      b->launch(grid, k & 1, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_per_step) ms_per_step[c] = ms / n_steps;
    if (ms / n_steps < best) {
      best = ms / n_steps;
      best_k = cand[c];
    }
  }
  // restore: states back into the buffers the descriptors name as current
  off = 0;
  for (auto* h : b->grids) {
    const Level& L = h->g.lv[0];
    cudaMemcpyAsync(L.f[L.cur], (char*)save + off, L.pop_bytes, cudaMemcpyDeviceToDevice, s);
    off += L.pop_bytes;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
  if (best_k != b->ctas_per_sm) {
    b->ctas_per_sm = best_k;
    b->drop_graphs();
  }
  if (chosen) *chosen = best_k;
  return LBM_OK;
}

}  // extern "C"
