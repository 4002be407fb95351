// noalloc.cu - conservation sums without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the mass / momentum sums: a solver loop that must never synchronise the
// device (cudaMalloc / cudaFree can block until all outstanding work is
// done), or an application whose device memory is handed out entirely by
// its own pool, where a library's private cudaMalloc would fail or fragment
// the pool.  lbm_conservation_noalloc serves them: the caller passes the
// populations and a 4-double output on the device; the per-CTA partial sums
// live in a fixed file-scope device array.
//
// That array is one per device that loads the library and stays allocated
// until the process exits.  Every call reuses it and it keeps the previous
// call's contents; each call writes every partial it later reads, so nothing
// needs clearing.  Two calls that run at the same time on the GPU (on
// different streams, or from different host threads) use the same array and
// race: order them on one stream.
#include <mutex>

#include "d3q19.cuh"
#include "grid.h"

namespace lbm {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_CHUNK = (int64_t)NA_THREADS * 64;  // voxels reduced per CTA
constexpr int NA_MAX_PARTIALS = 4096;                    // => at most 67,108,864 voxels
constexpr int64_t NA_MAX_VOXELS = NA_CHUNK * NA_MAX_PARTIALS;

static __device__ __align__(256) double g_noalloc_partials[NA_MAX_PARTIALS * 4];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int S>
__global__ void __launch_bounds__(NA_THREADS) na_partial(const void* f, int64_t n,
                                                         const uint8_t* flags, double* partials) {
  using T = typename Codec<S>::T;
  const T* in = (const T*)f;
  double acc[4] = {0, 0, 0, 0};
  const int64_t v0 = (int64_t)blockIdx.x * NA_CHUNK;
  int64_t v1 = v0 + NA_CHUNK;
  if (v1 > n) v1 = n;
  for (int64_t v = v0 + threadIdx.x; v < v1; v += NA_THREADS) {
    if (flags && !type_updated(flag_type(flags[v]))) continue;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double fi = Codec<S>::abs_d(in[(int64_t)i * n + v], i);
      acc[0] += fi;
      if (cx(i)) acc[1] += cx(i) * fi;
      if (cy(i)) acc[2] += cy(i) * fi;
      if (cz(i)) acc[3] += cz(i) * fi;
    }
  }
  __shared__ double sh[NA_THREADS / 32][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double w = na_warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w][threadIdx.x];
    partials[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(NA_THREADS) na_final(const double* partials, int np,
                                                       double* out4) {
  double acc[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < np; p += NA_THREADS)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += partials[p * 4 + k];
  __shared__ double sh[NA_THREADS / 32][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double w = na_warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w][threadIdx.x];
    out4[threadIdx.x] = t;
  }
}

// Device address of the partials array, looked up once per device with that
// device current (the host-side symbol is only a stand-in, never a device
// address).
constexpr int NA_MAX_DEVICES = 64;
static double* g_partials_addr[NA_MAX_DEVICES];
static std::once_flag g_partials_once[NA_MAX_DEVICES];
static cudaError_t g_partials_err[NA_MAX_DEVICES];

static lbm_status partials_address(double** out) {
  int dev = 0;
  LBM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(LBM_ERR_UNSUPPORTED, "device ordinal >= 64");
  std::call_once(g_partials_once[dev], [dev] {
    void* p = nullptr;
    g_partials_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_partials);
    g_partials_addr[dev] = (double*)p;
  });
  if (g_partials_err[dev] != cudaSuccess) return cuda_fail(g_partials_err[dev], "cudaGetSymbolAddress");
  *out = g_partials_addr[dev];
  return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_conservation_noalloc(const void* f, int storage, int64_t n_voxels,
                                               const uint8_t* flags, double* out_mass_mom,
                                               void* stream) {
  set_error("");
  if (!f || !out_mass_mom) return fail(LBM_ERR_INVALID, "NULL argument");
  if (storage < LBM_STORAGE_F32 || storage > LBM_STORAGE_BF16)
    return fail(LBM_ERR_INVALID, "unknown storage");
  if (n_voxels <= 0) return fail(LBM_ERR_INVALID, "n_voxels must be positive");
  if (n_voxels > NA_MAX_VOXELS)
    return fail(LBM_ERR_INVALID, "n_voxels exceeds the no-allocation limit of 67,108,864 voxels");
  double* partials = nullptr;
  lbm_status st = partials_address(&partials);
  if (st) return st;
  const int np = (int)((n_voxels + NA_CHUNK - 1) / NA_CHUNK);
  cudaStream_t s = (cudaStream_t)stream;
  switch (storage) {
    case LBM_STORAGE_F32: na_partial<S_F32><<<np, NA_THREADS, 0, s>>>(f, n_voxels, flags, partials); break;
    case LBM_STORAGE_F16: na_partial<S_F16><<<np, NA_THREADS, 0, s>>>(f, n_voxels, flags, partials); break;
    default: na_partial<S_BF16><<<np, NA_THREADS, 0, s>>>(f, n_voxels, flags, partials); break;
  }
  na_final<<<1, NA_THREADS, 0, s>>>(partials, np, out_mass_mom);
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}
