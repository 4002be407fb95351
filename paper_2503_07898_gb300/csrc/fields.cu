// fields.cu - layout-generic kernels: FP64 equilibrium initialisation,
// moments, FP64 population decode and the conservation reduction.
//
// A voxel (x, y, z) of a level's virtual box maps to storage as
//   dense : index(pop) = pop * N + v,                 v = x + nx (y + ny z)
//   sparse: index(pop) = (b * Q + pop) * E^3 + l,     b = block id from the
//           virtual block map, l = lx + E (ly + E lz)
#include "d3q19.cuh"
#include "grid.h"

namespace lbm {
namespace LBM_LNS {

struct LevelDev {
  int nx, ny, nz, E, nbx, nby, nbz;
  int64_t N;  // dense: voxels; sparse: slots
  const uint8_t* flags;  // dense: per voxel (may be null); sparse: per slot
  const int32_t* bmap;
};

static LevelDev level_dev(const Level& L) {
  LevelDev d;
  d.nx = L.nx;
  d.ny = L.ny;
  d.nz = L.nz;
  d.E = L.E;
  d.nbx = L.nbx;
  d.nby = L.nby;
  d.nbz = L.nbz;
  d.N = L.n_slots;
  d.flags = L.flags_d;
  d.bmap = L.bmap_d;
  return d;
}

// Storage base / stride of a virtual-box voxel; false if no storage exists.
__device__ __forceinline__ bool locate(const LevelDev& d, int x, int y, int z, int64_t& base,
                                       int64_t& stride, uint8_t& flag) {
  if (d.E == 0) {
    const int64_t v = x + (int64_t)d.nx * (y + (int64_t)d.ny * z);
    base = v;
    stride = d.N;
    flag = d.flags ? d.flags[v] : (uint8_t)0;
    return true;
  }
  const int E = d.E;
  const int bx = x / E, by = y / E, bz = z / E;
  const int b = d.bmap[bx + d.nbx * (by + d.nby * bz)];
  if (b < 0) return false;
  const int l = (x - bx * E) + E * ((y - by * E) + E * (z - bz * E));
  const int64_t E3 = (int64_t)E * E * E;
  base = (int64_t)b * Q * E3 + l;
  stride = E3;
  flag = d.flags[(int64_t)b * E3 + l];
  return true;
}

template <int S>
__global__ void k_init_eq(LevelDev d, void* f, const double* rho, const double* u) {
  using T = typename Codec<S>::T;
  const int64_t n = (int64_t)d.nx * d.ny * d.nz;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % d.nx);
    const int y = (int)((v / d.nx) % d.ny);
    const int z = (int)(v / ((int64_t)d.nx * d.ny));
    int64_t base, stride;
    uint8_t fl;
    if (!locate(d, x, y, z, base, stride, fl)) continue;
    if (!type_updated(flag_type(fl))) continue;
    const double r = rho ? rho[v] : 1.0;
    const double ux = u ? u[v] : 0.0, uy = u ? u[n + v] : 0.0, uz = u ? u[2 * n + v] : 0.0;
    T* out = (T*)f;
#pragma unroll
    for (int i = 0; i < Q; ++i) out[base + i * stride] = Codec<S>::from_double(feq_d(i, r, ux, uy, uz), i);
  }
}

template <int S>
__global__ void k_moments(LevelDev d, const void* f, double* rho, double* u) {
  using T = typename Codec<S>::T;
  const int64_t n = (int64_t)d.nx * d.ny * d.nz;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % d.nx);
    const int y = (int)((v / d.nx) % d.ny);
    const int z = (int)(v / ((int64_t)d.nx * d.ny));
    int64_t base, stride;
    uint8_t fl;
    double r = nan, ux = nan, uy = nan, uz = nan;
    if (locate(d, x, y, z, base, stride, fl) && type_updated(flag_type(fl))) {
      const T* in = (const T*)f;
      double m = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double fi = Codec<S>::abs_d(in[base + i * stride], i);
        m += fi;
        jx += cx(i) * fi;
        jy += cy(i) * fi;
        jz += cz(i) * fi;
      }
      r = m;
      ux = jx / m;
      uy = jy / m;
      uz = jz / m;
    }
    if (rho) rho[v] = r;
    if (u) {
      u[v] = ux;
      u[n + v] = uy;
      u[2 * n + v] = uz;
    }
  }
}

template <int S>
__global__ void k_decode(LevelDev d, const void* f, double* dst) {
  using T = typename Codec<S>::T;
  const int64_t n = (int64_t)d.nx * d.ny * d.nz;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % d.nx);
    const int y = (int)((v / d.nx) % d.ny);
    const int z = (int)(v / ((int64_t)d.nx * d.ny));
    int64_t base, stride;
    uint8_t fl;
    const bool ok = locate(d, x, y, z, base, stride, fl) && type_updated(flag_type(fl));
    const T* in = (const T*)f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      dst[i * n + v] = ok ? Codec<S>::abs_d(in[base + i * stride], i) : nan;
  }
}

// ---------------------------------------------------------------- reduction
// Pass 1: every CTA reduces a fixed, grid-strided set of slots to 4 doubles
// (warp shuffles, then shared memory) and writes them to partials[cta].
// Pass 2: one CTA adds the partials in a fixed order.  The result does not
// depend on scheduling, so repeated calls give bit-identical sums.
constexpr int RED_THREADS = 256;
constexpr int RED_CTAS = kRedCtas;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int S>
__global__ void __launch_bounds__(RED_THREADS) k_cons_partial(LevelDev d, const void* f,
                                                              double weight, double* partials) {
  using T = typename Codec<S>::T;
  const T* in = (const T*)f;
  double acc[4] = {0, 0, 0, 0};
  const int64_t E3 = d.E ? (int64_t)d.E * d.E * d.E : 1;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < d.N;
       s += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t fl = d.flags ? d.flags[s] : (uint8_t)0;
    if (!type_updated(flag_type(fl))) continue;
    int64_t base, stride;
    if (d.E == 0) {
      base = s;
      stride = d.N;
    } else {
      const int64_t b = s / E3;
      base = b * Q * E3 + (s - b * E3);
      stride = E3;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double fi = Codec<S>::abs_d(in[base + i * stride], i);
      acc[0] += fi;
      if (cx(i)) acc[1] += cx(i) * fi;
      if (cy(i)) acc[2] += cy(i) * fi;
      if (cz(i)) acc[3] += cz(i) * fi;
    }
  }
  __shared__ double sh[RED_THREADS / 32][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double w = warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int w = 0; w < RED_THREADS / 32; ++w) t += sh[w][threadIdx.x];
    partials[blockIdx.x * 4 + threadIdx.x] = t * weight;
  }
}

__global__ void __launch_bounds__(RED_THREADS) k_cons_final(const double* partials, int n,
                                                            double* out4) {
  double acc[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < n; p += blockDim.x)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += partials[p * 4 + k];
  __shared__ double sh[RED_THREADS / 32][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double w = warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int w = 0; w < RED_THREADS / 32; ++w) t += sh[w][threadIdx.x];
    out4[threadIdx.x] = t;
  }
}

// ------------------------------------------------------------------ launchers
static unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (unsigned)b;
}

lbm_status launch_init_equilibrium(Grid& g, Level& L, const double* rho, const double* u,
                                   cudaStream_t s) {
  const LevelDev d = level_dev(L);
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  const unsigned nb = grid_for(n, 256);
  switch (g.phys.storage) {
    case S_F32: k_init_eq<S_F32><<<nb, 256, 0, s>>>(d, L.f[L.cur], rho, u); break;
    case S_F16: k_init_eq<S_F16><<<nb, 256, 0, s>>>(d, L.f[L.cur], rho, u); break;
    default: k_init_eq<S_BF16><<<nb, 256, 0, s>>>(d, L.f[L.cur], rho, u); break;
  }
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}

lbm_status launch_moments(Grid& g, Level& L, double* rho, double* u, cudaStream_t s) {
  const LevelDev d = level_dev(L);
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  const unsigned nb = grid_for(n, 256);
  switch (g.phys.storage) {
    case S_F32: k_moments<S_F32><<<nb, 256, 0, s>>>(d, L.f[L.cur], rho, u); break;
    case S_F16: k_moments<S_F16><<<nb, 256, 0, s>>>(d, L.f[L.cur], rho, u); break;
    default: k_moments<S_BF16><<<nb, 256, 0, s>>>(d, L.f[L.cur], rho, u); break;
  }
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}

lbm_status launch_decode_f64(Grid& g, Level& L, double* dst, cudaStream_t s) {
  const LevelDev d = level_dev(L);
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  const unsigned nb = grid_for(n, 256);
  switch (g.phys.storage) {
    case S_F32: k_decode<S_F32><<<nb, 256, 0, s>>>(d, L.f[L.cur], dst); break;
    case S_F16: k_decode<S_F16><<<nb, 256, 0, s>>>(d, L.f[L.cur], dst); break;
    default: k_decode<S_BF16><<<nb, 256, 0, s>>>(d, L.f[L.cur], dst); break;
  }
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}

lbm_status launch_conservation(Grid& g, double* out4, cudaStream_t s) {
  int np = 0;
  for (int l = 0; l < g.n_levels; ++l) {
    Level& L = g.lv[l];
    const LevelDev d = level_dev(L);
    unsigned nb = (unsigned)((L.n_slots + RED_THREADS - 1) / RED_THREADS);
    if (nb > (unsigned)RED_CTAS) nb = RED_CTAS;
    if (nb < 1) nb = 1;
    const double w = (double)(1LL << (3 * l));  // 8^l volume weight
    double* part = g.partials_d + (size_t)np * 4;
    switch (g.phys.storage) {
      case S_F32: k_cons_partial<S_F32><<<nb, RED_THREADS, 0, s>>>(d, L.f[L.cur], w, part); break;
      case S_F16: k_cons_partial<S_F16><<<nb, RED_THREADS, 0, s>>>(d, L.f[L.cur], w, part); break;
      default: k_cons_partial<S_BF16><<<nb, RED_THREADS, 0, s>>>(d, L.f[L.cur], w, part); break;
    }
    np += (int)nb;
  }
  k_cons_final<<<1, RED_THREADS, 0, s>>>(g.partials_d, np, out4);
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}

}  // namespace LBM_LNS
}  // namespace lbm
