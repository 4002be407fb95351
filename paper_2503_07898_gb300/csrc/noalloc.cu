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
//
// The buffer may hold D3Q19 or D3Q27 populations (the caller says which);
// the kernels read the lattice's Q arrays and, for 16-bit storage, add back
// that lattice's weights.
#include <mutex>

#include "d3q19.cuh"
#include "grid.h"

namespace lbm {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_CHUNK = (int64_t)NA_THREADS * 64;  // voxels reduced per CTA
constexpr int NA_MAX_PARTIALS = 4096;                    // => at most 67,108,864 voxels
constexpr int64_t NA_MAX_VOXELS = NA_CHUNK * NA_MAX_PARTIALS;

static __device__ __align__(256) double g_noalloc_partials[NA_MAX_PARTIALS * 4];

// Lattice weights of D3Q19 (1/3, 1/18, 1/36) and D3Q27 (8/27, 2/27, 1/54,
// 1/216) in the library's velocity order (rest, 6 axes, 12 edges, 8 corners).
template <int QL>
__host__ __device__ constexpr double na_weight(int i) {
  return QL == 19 ? (i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0))
                  : (i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0)));
}

// Absolute population f_i in FP64 from the stored value (F32: f_i itself;
// F16 / BF16: f_i - w_i).
template <int S, int QL>
__device__ __forceinline__ double na_abs(const void* f, int64_t idx, int i) {
  if constexpr (S == S_F32) return (double)static_cast<const float*>(f)[idx];
  else if constexpr (S == S_F16)
    return na_weight<QL>(i) + (double)__half2float(static_cast<const __half*>(f)[idx]);
  else return na_weight<QL>(i) + (double)__bfloat162float(static_cast<const __nv_bfloat16*>(f)[idx]);
}

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int S, int QL>
__global__ void __launch_bounds__(NA_THREADS) na_partial(const void* f, int64_t n,
                                                         const uint8_t* flags, double* partials) {
  double acc[4] = {0, 0, 0, 0};
  const int64_t v0 = (int64_t)blockIdx.x * NA_CHUNK;
  int64_t v1 = v0 + NA_CHUNK;
  if (v1 > n) v1 = n;
  for (int64_t v = v0 + threadIdx.x; v < v1; v += NA_THREADS) {
    if (flags && !type_updated(flag_type(flags[v]))) continue;
#pragma unroll
    for (int i = 0; i < QL; ++i) {
      const double fi = na_abs<S, QL>(f, (int64_t)i * n + v, i);
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

// Device address of the partials array, looked up per device with that
// device current (the host-side symbol is only a stand-in, never a device
// address).  A successful lookup is kept; a failed one is retried on the
// next call.
constexpr int NA_MAX_DEVICES = 64;
static std::mutex g_partials_mutex;
static double* g_partials_addr[NA_MAX_DEVICES];

static lbm_status partials_address(int dev, double** out) {
  if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(LBM_ERR_UNSUPPORTED, "device ordinal >= 64");
  std::lock_guard<std::mutex> lock(g_partials_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return LBM_OK;
}

// A pointer the kernels may dereference: device (or managed) memory, and
// device memory of the current device.  Host and unregistered pointers are
// refused before any launch.
static lbm_status check_device_pointer(const void* p, int dev, const char* what) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_ERR_INVALID, std::string(what) + " is not a CUDA pointer");
  }
  if (a.type == cudaMemoryTypeManaged) return LBM_OK;
  if (a.type != cudaMemoryTypeDevice)
    return fail(LBM_ERR_INVALID, std::string(what) + " is not device memory");
  if (a.device != dev)
    return fail(LBM_ERR_INVALID, std::string(what) + " is on another device");
  return LBM_OK;
}

template <int QL>
static void launch_partials(int storage, int np, const void* f, int64_t n, const uint8_t* flags,
                            double* partials, cudaStream_t s) {
  switch (storage) {
    case LBM_STORAGE_F32: na_partial<S_F32, QL><<<np, NA_THREADS, 0, s>>>(f, n, flags, partials); break;
    case LBM_STORAGE_F16: na_partial<S_F16, QL><<<np, NA_THREADS, 0, s>>>(f, n, flags, partials); break;
    default: na_partial<S_BF16, QL><<<np, NA_THREADS, 0, s>>>(f, n, flags, partials); break;
  }
}

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_conservation_noalloc(const void* f, int storage, int lattice,
                                               int64_t n_voxels, const uint8_t* flags,
                                               double* out_mass_mom, void* stream) {
  set_error("");
  if (!f || !out_mass_mom) return fail(LBM_ERR_INVALID, "NULL argument");
  if (storage < LBM_STORAGE_F32 || storage > LBM_STORAGE_BF16)
    return fail(LBM_ERR_INVALID, "unknown storage");
  if (lattice == 0) lattice = 19;
  if (lattice != 19 && lattice != 27) return fail(LBM_ERR_INVALID, "lattice must be 19 or 27");
  if (n_voxels <= 0) return fail(LBM_ERR_INVALID, "n_voxels must be positive");
  if (n_voxels > NA_MAX_VOXELS)
    return fail(LBM_ERR_INVALID, "n_voxels exceeds the no-allocation limit of 67,108,864 voxels");
  int dev = 0;
  LBM_CUDA(cudaGetDevice(&dev));
  lbm_status st = check_device_pointer(f, dev, "f");
  if (!st) st = check_device_pointer(out_mass_mom, dev, "out_mass_mom");
  if (!st && flags) st = check_device_pointer(flags, dev, "flags");
  if (st) return st;
  double* partials = nullptr;
  st = partials_address(dev, &partials);
  if (st) return st;
  const int np = (int)((n_voxels + NA_CHUNK - 1) / NA_CHUNK);
  cudaStream_t s = (cudaStream_t)stream;
  if (lattice == 19) launch_partials<19>(storage, np, f, n_voxels, flags, partials, s);
  else launch_partials<27>(storage, np, f, n_voxels, flags, partials, s);
  na_final<<<1, NA_THREADS, 0, s>>>(partials, np, out_mass_mom);
  LBM_CUDA(cudaGetLastError());
  return LBM_OK;
}
