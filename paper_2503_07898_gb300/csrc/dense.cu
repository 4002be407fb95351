// dense.cu - fused pull stream-and-collide kernels on dense grids.
//
// Disaggregated dense layout (Sec. 3 and Sec. 6.1, adapted to one GPU): the
// voxels needing the register-heavy regularized boundary (Sec. 6.2) form
// the boundary group G_b; every other voxel is in G_nb.  Populations are
// SoA, index pop * N + v with v = x + nx (y + ny z).  When G_b is the last
// n_b voxel ids (a lid on the top plane) both groups are contiguous ranges
// (Table 2, "Disag - Mem": direct indexing, no extra storage) and the
// interior kernel runs without any per-voxel flag.  Otherwise a per-voxel
// 32-bit wall mask tells the interior kernel which pull sources bounce back
// and which voxels to skip.
//
// Kernels
//   dense_interior<S, COLL>  G_nb: pull + bounce-back + BGK / REG collision
//                            (2Q live values; bounded to 64 registers)
//   dense_boundary<S>        G_b : pull + regularized node (3Q live values)
//   dense_monolithic<S,COLL> the paper's naive kernel (Sec. 4): every voxel,
//                            per-voxel branch on its flag, boundary values
//                            read from a full-domain array
#include "dense.cuh"
#include "d3q19.cuh"
#include "grid.h"

namespace lbm {
namespace LBM_LNS {

// Per-population base addresses of the interior kernel, passed as kernel
// parameters: a pull source or a store target is then one multiply-add of a
// 32-bit (or 64-bit) voxel offset onto a constant-bank base.  in[I] points
// at population I of the input shifted by -c_x(I) elements, so that the
// source of voxel v is in[I][v + row offset of (c_y, c_z)]; out[I] at
// population I of the output.
struct DensePops {
  const void* in[Q];
  void* out[Q];
};

template <int S, int COLL, class IDX>
__global__ void __launch_bounds__(256, S == S_F32 ? 4 : 5) dense_interior(DenseArgs a, DensePops p) {
  using T = typename Codec<S>::T;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const int64_t v = x + (int64_t)a.nx * (y + (int64_t)a.ny * z);
  if (v >= a.vend) return;
  float g[Q];
  uint32_t wm = 0;
  if (a.wmask) {
    wm = a.wmask[v];
    if (wm & (WM_SKIP | WM_REG)) return;
  }
  // warp-uniform choice: a warp holds one (y, z) row.  16-bit storage, whose
  // kernel is bound by instruction issue, takes the select-free lean pull
  // and the per-population bases; FP32, bound by DRAM, keeps one offset
  // and selects per population (measured 0.2 % faster for D3Q19, 1 % for
  // D3Q27)
  if (lean_row(a, y, z)) {
    if constexpr (S == S_F32) {
      if (wm) pull_row_interior<S, IDX, true>((const T*)a.fin, a, x, y, z, (IDX)v, wm, g);
      else pull_row_interior<S, IDX, false>((const T*)a.fin, a, x, y, z, (IDX)v, 0u, g);
    } else {
      pull_lean<S, IDX>(a, x, y, z, (IDX)v, wm, g, [&](auto ic, IDX o) {
        return reinterpret_cast<const T*>(p.in[decltype(ic)::value])[o];
      });
    }
  } else {
    pull_all<S>((const T*)a.fin, a, x, y, z, v, wm, g);
  }
  collide<COLL>(g, a.omega);
  if constexpr (S == S_F32) {
    T* __restrict__ fout = (T*)a.fout;
    const IDX N = (IDX)a.N;
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      fout[(IDX)I * N + (IDX)v] = Codec<S>::template store<I>(g[I]);
    });
  } else {
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      reinterpret_cast<T*>(p.out[I])[(IDX)v] = Codec<S>::template store<I>(g[I]);
    });
  }
}

// ------------------------------------------------------------------------
// Vectorized interior kernel for grids whose walls are only box sides.
// A thread owns V consecutive voxels along x and moves every population as
// one aligned vector (V * sizeof(T) = 16 bytes: 4 FP32 or 8 FP16 / BF16
// values), so a warp reads and writes 512 contiguous bytes per population.
// A pull with c_x = +1 needs the element left of the vector: it comes from
// lane - 1 by a warp shuffle; lane 0 (and the thread at x = 0) fetches it
// itself, wrapping or bouncing back at the box side.  c_x = -1 mirrors this
// with lane + 1.  Rows whose source (y - c_y, z - c_z) leaves a non-periodic
// box side bounce back as a whole (warp-uniform).  Loads and stores use the
// streaming cache hint: every population value is read exactly once.
template <class T, int V> struct alignas(sizeof(T) * V) PVec { T e[V]; };

template <class T, int V>
__device__ __forceinline__ PVec<T, V> ld_vec(const T* p) {
  PVec<T, V> r;
  if constexpr (sizeof(T) * V == 16) {
    uint4 u = __ldcs(reinterpret_cast<const uint4*>(p));
    memcpy(&r, &u, 16);
  } else if constexpr (sizeof(T) * V == 4) {
    unsigned int u = __ldcs(reinterpret_cast<const unsigned int*>(p));
    memcpy(&r, &u, 4);
  } else {
    uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
    memcpy(&r, &u, 8);
  }
  return r;
}

template <class T, int V>
__device__ __forceinline__ void st_vec(T* p, const PVec<T, V>& r) {
  if constexpr (sizeof(T) * V == 16) {
    uint4 u;
    memcpy(&u, &r, 16);
    __stcs(reinterpret_cast<uint4*>(p), u);
  } else if constexpr (sizeof(T) * V == 4) {
    unsigned int u;
    memcpy(&u, &r, 4);
    __stcs(reinterpret_cast<unsigned int*>(p), u);
  } else {
    uint2 u;
    memcpy(&u, &r, 8);
    __stcs(reinterpret_cast<uint2*>(p), u);
  }
}

constexpr int VEC_ROWS = 4;  // warps (rows along y) per CTA

template <int S, int COLL, int V>
__global__ void __launch_bounds__(32 * VEC_ROWS) dense_interior_vec(DenseArgs a) {
  using T = typename Codec<S>::T;
  using Vt = PVec<T, V>;
  const T* __restrict__ fin = (const T*)a.fin;
  T* __restrict__ fout = (T*)a.fout;
  const int lane = threadIdx.x;
  const int x = (blockIdx.x * 32 + lane) * V;
  const int y = blockIdx.y * VEC_ROWS + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= a.ny) return;  // uniform per warp
  const bool active = x < a.nx;
  const int64_t v = x + (int64_t)a.nx * (y + (int64_t)a.ny * z);
  const bool last = lane == 31 || x + V >= a.nx;  // the next lane holds no voxel of this row
  Vt f[Q];
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int ys = y - cy(I), zs = z - cz(I);
    bool rwall = false;
    if constexpr (cy(I) != 0) {
      if (ys < 0 || ys >= a.ny) {
        if (a.py) ys += ys < 0 ? a.ny : -a.ny; else rwall = true;
      }
    }
    if constexpr (cz(I) != 0) {
      if (zs < 0 || zs >= a.nz) {
        if (a.pz) zs += zs < 0 ? a.nz : -a.nz; else rwall = true;
      }
    }
    if (rwall) {
      if (active) f[I] = ld_vec<T, V>(fin + (int64_t)opp(I) * a.N + v);
      return;
    }
    const T* src = fin + (int64_t)I * a.N + (int64_t)a.nx * (ys + (int64_t)a.ny * zs);
    Vt A;
    if (active) A = ld_vec<T, V>(src + x);
    if constexpr (cx(I) == 0) {
      f[I] = A;
    } else if constexpr (cx(I) == 1) {
      T left = __shfl_up_sync(0xffffffffu, A.e[V - 1], 1);
      if (active && lane == 0) {
        if (x > 0) left = src[x - 1];
        else left = a.px ? src[a.nx - 1] : fin[(int64_t)opp(I) * a.N + v];
      }
      f[I].e[0] = left;
#pragma unroll
      for (int k = 1; k < V; ++k) f[I].e[k] = A.e[k - 1];
    } else {
      T right = __shfl_down_sync(0xffffffffu, A.e[0], 1);
      if (active && last) {
        if (x + V < a.nx) right = src[x + V];
        else right = a.px ? src[0] : fin[(int64_t)opp(I) * a.N + v + V - 1];
      }
#pragma unroll
      for (int k = 0; k < V - 1; ++k) f[I].e[k] = A.e[k + 1];
      f[I].e[V - 1] = right;
    }
  });
  if (!active) return;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    float g[Q];
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      g[I] = Codec<S>::template load<I>(f[I].e[k]);
    });
    collide<COLL>(g, a.omega);
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      f[I].e[k] = Codec<S>::template store<I>(g[I]);
    });
  }
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    st_vec<T, V>(fout + (int64_t)I * a.N + v, f[I]);
  });
}

template <int S>
__global__ void __launch_bounds__(128) dense_boundary(DenseArgs a) {
  using T = typename Codec<S>::T;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nlist) return;
  const int64_t v = a.list ? (int64_t)a.list[t] : a.v0 + t;
  const int64_t plane = (int64_t)a.nx * a.ny;
  const int z = (int)(v / plane);
  const int64_t r = v - (int64_t)z * plane;
  const int y = (int)(r / a.nx);
  const int x = (int)(r - (int64_t)y * a.nx);
  const uint32_t wm = a.wmask ? a.wmask[v] : 0u;
  const uint8_t fl = a.flags[v];
  float g[Q];
  pull_all<S>((const T*)a.fin, a, x, y, z, v, wm, g);
  regularized_node(g, flag_type(fl), flag_normal(fl), a.bc[t], a.omega);
  store_all<S>((T*)a.fout, a, v, g);
}

template <int S, int COLL>
__global__ void __launch_bounds__(256) dense_monolithic(DenseArgs a) {
  using T = typename Codec<S>::T;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const int64_t v = x + (int64_t)a.nx * (y + (int64_t)a.ny * z);
  const uint8_t fl = a.flags ? a.flags[v] : (uint8_t)0;
  const int type = flag_type(fl);
  if (!type_updated(type)) return;
  const uint32_t wm = a.wmask ? (a.wmask[v] & ~WM_REG) : 0u;
  float g[Q];
  pull_all<S>((const T*)a.fin, a, x, y, z, v, wm, g);
  if (type_regularized(type)) {
    regularized_node(g, type, flag_normal(fl), a.bc[v], a.omega);
  } else {
    collide<COLL>(g, a.omega);
  }
  store_all<S>((T*)a.fout, a, v, g);
}

template <int S, int COLL>
static lbm_status dense_step_t(Grid& g, Level& L, cudaStream_t s) {
  DenseArgs a{};
  a.fin = L.f[L.cur];
  a.fout = L.f[L.cur ^ 1];
  a.nx = L.nx;
  a.ny = L.ny;
  a.nz = L.nz;
  a.N = L.n_slots;
  a.px = g.phys.periodic[0];
  a.py = g.phys.periodic[1];
  a.pz = g.phys.periodic[2];
  a.wmask = L.wmask_d;
  a.flags = L.flags_d;
  a.omega = (float)(1.0 / g.phys.tau);
  const dim3 blk(32, 8);
  const int gx = (L.nx + 31) / 32, gy = (L.ny + 7) / 8;
  if (g.phys.schedule == LBM_SCHEDULE_MONOLITHIC) {
    a.bc = L.bc_full_d;
    const int pr = prof_begin(g, s, "dense_monolithic", L.n_updated);
    dense_monolithic<S, COLL><<<dim3(gx, gy, L.nz), blk, 0, s>>>(a);
    prof_end(g, s, pr);
  } else {
    const int64_t plane = (int64_t)L.nx * L.ny;
    a.vend = L.dense_reg_tail ? L.n_slots - L.n_reg : L.n_slots;
    const int zc = (int)((a.vend + plane - 1) / plane);
    // vector widths: 16 bytes (default) or 8 bytes; scalar when the grid has
    // per-voxel walls, an x extent that is not a multiple of V, or a
    // boundary group that is not a whole number of top planes
    constexpr int V16 = 16 / (int)sizeof(typename Codec<S>::T);
    constexpr int V8 = 8 / (int)sizeof(typename Codec<S>::T);
    constexpr int V4 = 4 / (int)sizeof(typename Codec<S>::T);  // 2 for 16-bit storage, else 1
    const int vw = L.variant == VARIANT_SCALAR ? 0
                   : L.variant == VARIANT_VEC8 ? V8
                   : L.variant == VARIANT_VEC4 ? (V4 >= 2 ? V4 : 0)
                                               : V16;
    const bool vec_ok = vw > 0 && !L.wmask_d && L.nx % vw == 0 && a.vend % plane == 0;
    // the boundary group (regularized voxels) runs beside the interior
    // kernel on the grid's high-priority group stream: both read the
    // previous state and write disjoint voxels
    const bool fork = L.n_reg > 0 && zc > 0;
    cudaStream_t sb = s;
    if (fork) {
      lbm_status st = group_fork(g, s, &sb);
      if (st) return st;
    }
    if (L.n_reg > 0) {
      a.bc = L.bc_grp_d;
      a.list = L.dense_reg_tail ? nullptr : L.reg_list_d;
      a.v0 = L.n_slots - L.n_reg;
      a.nlist = L.n_reg;
      const int pr = prof_begin(g, sb, "dense_boundary", L.n_reg);
      dense_boundary<S><<<(unsigned)((L.n_reg + 127) / 128), 128, 0, sb>>>(a);
      prof_end(g, sb, pr);
    }
    if (zc > 0 && vec_ok) {
      const int pr = prof_begin(g, s, "dense_interior_vec", L.n_updated - L.n_reg);
      const dim3 vb(32, VEC_ROWS), vg((L.nx + 32 * vw - 1) / (32 * vw), (L.ny + VEC_ROWS - 1) / VEC_ROWS, zc);
      bool launched = false;
      if constexpr (V4 >= 2) {
        if (vw == V4) {
          dense_interior_vec<S, COLL, V4><<<vg, vb, 0, s>>>(a);
          launched = true;
        }
      }
      if (!launched) {
        if (vw == V16) dense_interior_vec<S, COLL, V16><<<vg, vb, 0, s>>>(a);
        else dense_interior_vec<S, COLL, V8><<<vg, vb, 0, s>>>(a);
      }
      prof_end(g, s, pr);
    } else if (zc > 0) {
      const int pr = prof_begin(g, s, "dense_interior", L.n_updated - L.n_reg);
      using T = typename Codec<S>::T;
      DensePops p;
      for (int i = 0; i < Q; ++i) {
        p.in[i] = (const T*)a.fin + ((int64_t)i * L.n_slots - cx(i));
        p.out[i] = (T*)a.fout + (int64_t)i * L.n_slots;
      }
      // 32-bit offsets while they fit: FP32 indexes every population from
      // the first (Q N elements); 16-bit offsets are per population and stay
      // below N + nx ny
      if ((S == S_F32 ? (int64_t)Q * L.n_slots : L.n_slots + (int64_t)L.nx * L.ny) < (1LL << 31))
        dense_interior<S, COLL, int32_t><<<dim3(gx, gy, zc), blk, 0, s>>>(a, p);
      else
        dense_interior<S, COLL, int64_t><<<dim3(gx, gy, zc), blk, 0, s>>>(a, p);
      prof_end(g, s, pr);
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

void dense_wall_mask(const Grid& g, const Level& L, std::vector<uint32_t>& wm) {
  const int* per = g.phys.periodic;
  const int n[3] = {L.nx, L.ny, L.nz};
  wm.assign((size_t)L.n_slots, 0u);
  for (int z = 0; z < L.nz; ++z)
    for (int y = 0; y < L.ny; ++y)
      for (int x = 0; x < L.nx; ++x) {
        const int64_t v = x + (int64_t)L.nx * (y + (int64_t)L.ny * z);
        const int t = flag_type(L.flags_h[(size_t)v]);
        uint32_t m = 0;
        if (!type_updated(t)) m |= WM_SKIP;
        if (type_regularized(t)) m |= WM_REG;
        for (int i = 1; i < Q; ++i) {
          int sc[3] = {x - cx(i), y - cy(i), z - cz(i)};
          bool wall = false;
          for (int a = 0; a < 3; ++a)
            if (sc[a] < 0 || sc[a] >= n[a]) {
              if (per[a]) sc[a] = (sc[a] + n[a]) % n[a];
              else wall = true;
            }
          if (!wall)
            wall = type_wall(flag_type(L.flags_h[(size_t)(sc[0] + (int64_t)L.nx * (sc[1] + (int64_t)L.ny * sc[2]))]));
          if (wall) m |= 1u << i;
        }
        wm[(size_t)v] = m;
      }
}

lbm_status dense_step(Grid& g, Level& L, cudaStream_t s) {
  const int st = g.phys.storage, co = g.phys.collision;
  if (st == S_F32) return co == C_BGK ? dense_step_t<S_F32, C_BGK>(g, L, s)
                                      : dense_step_t<S_F32, C_REG>(g, L, s);
  if (st == S_F16) return co == C_BGK ? dense_step_t<S_F16, C_BGK>(g, L, s)
                                      : dense_step_t<S_F16, C_REG>(g, L, s);
  return co == C_BGK ? dense_step_t<S_BF16, C_BGK>(g, L, s) : dense_step_t<S_BF16, C_REG>(g, L, s);
}

}  // namespace LBM_LNS
}  // namespace lbm
