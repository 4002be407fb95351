// closure.cu - learned closure: dataset generation, training and inference
// entry points (kernels for the network itself live in closure.cuh).
//
// Training data are made by the solver: a fine periodic dense run is
// box-filtered by r^3 (mean populations), the filtered populations are
// streamed one coarse step (what a coarse voxel pulls) and turned into
// features; the target is the least-squares eddy viscosity over each coarse
// voxel's 3^3 neighbourhood, d_tau = 3 nu_t with
// nu_t = - sum tau_sgs_dev : S / sum 2 rho S : S,
// tau_sgs = mean(rho u u) - rho u_bar u_bar and S the central-difference strain
// of u_bar, clamped to [-(tau_c - 1/2) + 1e-3, 1/2].
// Training is plain FP32 on CUDA cores (the batch GEMMs are small): forward,
// backward, Adam, deterministic loop orders; minibatches are drawn with the
// SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014) on the counter
// step * batch + b.
#include <cmath>
#include <vector>

#include "closure.cuh"
#include "d3q19.cuh"
#include "grid.h"

namespace lbm {

// parameter offsets in the flat FP32 vector
constexpr int P_W1 = 0, P_B1 = 1024, P_W2 = 1088, P_B2 = 5184, P_W3 = 5248, P_B3 = 5312;

// ------------------------------------------------------------ inference checks

__global__ void __launch_bounds__(256) k_mlp_forward_bf16(const ClosureParams* p, const float* X,
                                                          int64_t n, float* y) {
  __shared__ ClosureSmem sm;
  __shared__ __nv_bfloat16 stage[8][32 * FSTAGE];
  closure_load_smem(sm, p);
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float x[MLP_IN];
#pragma unroll
  for (int k = 0; k < MLP_IN; ++k) x[k] = i < n ? X[i * MLP_IN + k] : 0.f;
  const float out = mlp_bf16_warp(x, sm, stage[threadIdx.x >> 5]);
  if (i < n) y[i] = out;
}

__global__ void k_mlp_forward_fp32(const float* th, const float* X, int64_t n, float* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[MLP_IN], h1[MLP_H];
  for (int k = 0; k < MLP_IN; ++k) x[k] = X[i * MLP_IN + k];
  for (int j = 0; j < MLP_H; ++j) {
    float z = th[P_B1 + j];
    for (int k = 0; k < MLP_IN; ++k) z += th[P_W1 + j * MLP_IN + k] * x[k];
    h1[j] = fmaxf(z, 0.f);
  }
  float out = th[P_B3];
  for (int j = 0; j < MLP_H; ++j) {
    float z = th[P_B2 + j];
    for (int k = 0; k < MLP_H; ++k) z += th[P_W2 + j * MLP_H + k] * h1[k];
    out += fmaxf(z, 0.f) * th[P_W3 + j];
  }
  y[i] = out;
}

// ------------------------------------------------------------------ training

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Gather (and normalise) one minibatch.
__global__ void k_gather(const float* X, const float* T, int64_t n, const int32_t* idx,
                         uint64_t seed, int64_t counter0, int B, const float* stats, float* Xb,
                         float* tb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int64_t i = idx ? (int64_t)idx[b] : (int64_t)(splitmix64(seed + (uint64_t)(counter0 + b)) % (uint64_t)n);
  for (int k = 0; k < MLP_IN; ++k)
    Xb[b * MLP_IN + k] = stats ? (X[i * MLP_IN + k] - stats[k]) / stats[MLP_IN + k] : X[i * MLP_IN + k];
  tb[b] = stats ? (T[i] - stats[2 * MLP_IN]) / stats[2 * MLP_IN + 1] : T[i];
}

// out[b][j] = act(sum_k in[b][k] W[j][k] + bias[j]); pre-activation kept.
__global__ void k_dense(const float* in, int K, const float* W, const float* bias, int OUT, int B,
                        bool relu, float* pre, float* act) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * OUT) return;
  const int b = t / OUT, j = t % OUT;
  float z = bias[j];
  for (int k = 0; k < K; ++k) z += in[b * K + k] * W[j * K + k];
  pre[t] = z;
  act[t] = relu ? fmaxf(z, 0.f) : z;
}

__global__ void k_loss(const float* y, const float* t, int B, float* dy, float* loss) {
  __shared__ float sh[256];
  float acc = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float r = y[b] - t[b];
    dy[b] = 2.f * r / (float)B;
    acc += r * r;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (float)B;
}

// gW[j][k] = sum_b dz[b][j] in[b][k]; gb[j] = sum_b dz[b][j]
__global__ void k_grad_w(const float* dz, const float* in, int OUT, int K, int B, float* gW,
                         float* gb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < OUT * K) {
    const int j = t / K, k = t % K;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dz[b * OUT + j] * in[b * K + k];
    gW[t] = s;
  } else if (t < OUT * K + OUT) {
    const int j = t - OUT * K;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dz[b * OUT + j];
    gb[j] = s;
  }
}

// dz[b][i] = (sum_j dnext[b][j] Wn[j][i]) * (z[b][i] > 0)
__global__ void k_back(const float* dnext, const float* Wn, int OUT2, const float* z, int OUT1,
                       int B, float* dz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * OUT1) return;
  const int b = t / OUT1, i = t % OUT1;
  float s = 0.f;
  for (int j = 0; j < OUT2; ++j) s += dnext[b * OUT2 + j] * Wn[j * OUT1 + i];
  dz[t] = z[t] > 0.f ? s : 0.f;
}

__global__ void k_adam(float* th, const float* g, float* m, float* v, int n, float lr, float c1,
                       float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mi = 0.9f * m[i] + 0.1f * g[i];
  const float vi = 0.999f * v[i] + 0.001f * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// Column statistics (mean, standard deviation) of features and targets.
__global__ void k_stats(const float* X, const float* T, int64_t n, float* stats) {
  const int c = blockIdx.x;  // 0..16 (16 = target)
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = c < MLP_IN ? X[i * MLP_IN + c] : T[i];
    a += v;
    b += v * v;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      s1[threadIdx.x] += s1[threadIdx.x + s];
      s2[threadIdx.x] += s2[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = s1[0] / (double)n;
    double var = s2[0] / (double)n - mean * mean;
    double sd = var > 0 ? sqrt(var) : 0.0;
    // constant column (the tau feature of a one-level set): a deviation below
    // 1e-6 of the mean's magnitude is rounding noise of the FP64 sums, and as
    // a scale it would blow up the folded first layer
    if (!(sd > 1e-30) || !(sd > 1e-6 * fabs(mean))) sd = 1.0;
    const int im = c < MLP_IN ? c : 2 * MLP_IN, is = c < MLP_IN ? MLP_IN + c : 2 * MLP_IN + 1;
    stats[im] = (float)mean;
    stats[is] = (float)sd;
  }
}

struct TrainBufs {
  float *Xb, *tb, *z1, *h1, *z2, *h2, *y, *dy, *dz2, *dz1, *loss;
};

// Loss and gradient of one (gathered) minibatch at th; grad gets 5313 values.
static void batch_grad(const float* th, const TrainBufs& t, int B, float* grad, cudaStream_t s) {
  const int T = 256;
  auto nb = [&](int64_t n) { return (unsigned)((n + T - 1) / T); };
  k_dense<<<nb((int64_t)B * MLP_H), T, 0, s>>>(t.Xb, MLP_IN, th + P_W1, th + P_B1, MLP_H, B, true, t.z1, t.h1);
  k_dense<<<nb((int64_t)B * MLP_H), T, 0, s>>>(t.h1, MLP_H, th + P_W2, th + P_B2, MLP_H, B, true, t.z2, t.h2);
  k_dense<<<nb(B), T, 0, s>>>(t.h2, MLP_H, th + P_W3, th + P_B3, 1, B, false, t.y, t.y);
  k_loss<<<1, 256, 0, s>>>(t.y, t.tb, B, t.dy, t.loss);
  k_grad_w<<<nb(MLP_H + 1), T, 0, s>>>(t.dy, t.h2, 1, MLP_H, B, grad + P_W3, grad + P_B3);
  k_back<<<nb((int64_t)B * MLP_H), T, 0, s>>>(t.dy, th + P_W3, 1, t.z2, MLP_H, B, t.dz2);
  k_grad_w<<<nb(MLP_H * MLP_H + MLP_H), T, 0, s>>>(t.dz2, t.h1, MLP_H, MLP_H, B, grad + P_W2, grad + P_B2);
  k_back<<<nb((int64_t)B * MLP_H), T, 0, s>>>(t.dz2, th + P_W2, MLP_H, t.z1, MLP_H, B, t.dz1);
  k_grad_w<<<nb(MLP_H * MLP_IN + MLP_H), T, 0, s>>>(t.dz1, t.Xb, MLP_H, MLP_IN, B, grad + P_W1, grad + P_B1);
}

struct DevBuf {
  void* p = nullptr;
  explicit DevBuf(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  float* f() const { return (float*)p; }
};

static bool alloc_train(int B, std::vector<DevBuf*>& keep, TrainBufs& t) {
  auto mk = [&](size_t n) -> float* {
    keep.push_back(new DevBuf(n * sizeof(float)));
    return keep.back()->f();
  };
  t.Xb = mk((size_t)B * MLP_IN);
  t.tb = mk(B);
  t.z1 = mk((size_t)B * MLP_H);
  t.h1 = mk((size_t)B * MLP_H);
  t.z2 = mk((size_t)B * MLP_H);
  t.h2 = mk((size_t)B * MLP_H);
  t.y = mk(B);
  t.dy = mk(B);
  t.dz2 = mk((size_t)B * MLP_H);
  t.dz1 = mk((size_t)B * MLP_H);
  t.loss = mk(1);
  for (auto* d : keep)
    if (!d->p) return false;
  return true;
}

// ------------------------------------------------------------------- dataset

struct DsArgs {
  const void* f;  // fine populations (dense SoA)
  int nx, ny, nz, r, cx_, cy_, cz_;  // fine dims, filter, coarse dims
  int64_t N;
  float* sbar;   // 19 x nc shifted filtered populations
  float* mom;    // 10 x nc: rho, j (3), mean(j_a j_b / rho) (6: xx yy zz xy xz yz)
  float* num;    // nc
  float* den;    // nc
};

template <int S>
__global__ void k_ds_filter(DsArgs a) {
  using T = typename Codec<S>::T;
  const int64_t nc = (int64_t)a.cx_ * a.cy_ * a.cz_;
  const int64_t X = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (X >= nc) return;
  const int Xx = (int)(X % a.cx_), Xy = (int)((X / a.cx_) % a.cy_), Xz = (int)(X / ((int64_t)a.cx_ * a.cy_));
  const T* f = (const T*)a.f;
  double sp[Q], m[10];
  for (int i = 0; i < Q; ++i) sp[i] = 0;
  for (int k = 0; k < 10; ++k) m[k] = 0;
  for (int dz = 0; dz < a.r; ++dz)
    for (int dy = 0; dy < a.r; ++dy)
      for (int dx = 0; dx < a.r; ++dx) {
        const int64_t v = (Xx * a.r + dx) + (int64_t)a.nx * ((Xy * a.r + dy) + (int64_t)a.ny * (Xz * a.r + dz));
        double rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const double fi = Codec<S>::abs_d(f[(int64_t)i * a.N + v], i);
          sp[i] += fi - wd(i);
          rho += fi;
          jx += cx(i) * fi;
          jy += cy(i) * fi;
          jz += cz(i) * fi;
        }
        m[0] += rho;
        m[1] += jx;
        m[2] += jy;
        m[3] += jz;
        m[4] += jx * jx / rho;
        m[5] += jy * jy / rho;
        m[6] += jz * jz / rho;
        m[7] += jx * jy / rho;
        m[8] += jx * jz / rho;
        m[9] += jy * jz / rho;
      }
  const double inv = 1.0 / ((double)a.r * a.r * a.r);
  for (int i = 0; i < Q; ++i) a.sbar[(int64_t)i * nc + X] = (float)(sp[i] * inv);
  for (int k = 0; k < 10; ++k) a.mom[(int64_t)k * nc + X] = (float)(m[k] * inv);
}

__device__ __forceinline__ int64_t cidx(const DsArgs& a, int x, int y, int z) {
  x = (x + a.cx_) % a.cx_;
  y = (y + a.cy_) % a.cy_;
  z = (z + a.cz_) % a.cz_;
  return x + (int64_t)a.cx_ * (y + (int64_t)a.cy_ * z);
}

__global__ void k_ds_features(DsArgs a, float tau, float* feats) {
  const int64_t nc = (int64_t)a.cx_ * a.cy_ * a.cz_;
  const int64_t X = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (X >= nc) return;
  const int x = (int)(X % a.cx_), y = (int)((X / a.cx_) % a.cy_), z = (int)(X / ((int64_t)a.cx_ * a.cy_));
  float s[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) s[i] = a.sbar[(int64_t)i * nc + cidx(a, x - cx(i), y - cy(i), z - cz(i))];
  float xf[MLP_IN];
  closure_features(s, tau, xf);
  for (int k = 0; k < MLP_IN; ++k) feats[X * MLP_IN + k] = xf[k];
}

__global__ void k_ds_numden(DsArgs a) {
  const int64_t nc = (int64_t)a.cx_ * a.cy_ * a.cz_;
  const int64_t X = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (X >= nc) return;
  const int x = (int)(X % a.cx_), y = (int)((X / a.cx_) % a.cy_), z = (int)(X / ((int64_t)a.cx_ * a.cy_));
  auto ub = [&](int b, int xx, int yy, int zz) {
    const int64_t i = cidx(a, xx, yy, zz);
    return (double)a.mom[(int64_t)(1 + b) * nc + i] / (double)a.mom[i];
  };
  double g[3][3];  // g[a][b] = d u_b / d x_a
  for (int b = 0; b < 3; ++b) {
    g[0][b] = 0.5 * (ub(b, x + 1, y, z) - ub(b, x - 1, y, z));
    g[1][b] = 0.5 * (ub(b, x, y + 1, z) - ub(b, x, y - 1, z));
    g[2][b] = 0.5 * (ub(b, x, y, z + 1) - ub(b, x, y, z - 1));
  }
  const double rb = a.mom[X];
  const double u[3] = {a.mom[1 * nc + X] / rb, a.mom[2 * nc + X] / rb, a.mom[3 * nc + X] / rb};
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  double t[3][3];
  for (int k = 0; k < 6; ++k) {
    const double v = (double)a.mom[(int64_t)(4 + k) * nc + X] - rb * u[pa[k]] * u[pb[k]];
    t[pa[k]][pb[k]] = v;
    t[pb[k]][pa[k]] = v;
  }
  const double tr = (t[0][0] + t[1][1] + t[2][2]) / 3.0;
  double num = 0, den = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double Sij = 0.5 * (g[i][j] + g[j][i]);
      num += (t[i][j] - (i == j ? tr : 0.0)) * Sij;
      den += Sij * Sij;
    }
  a.num[X] = (float)num;
  a.den[X] = (float)(2.0 * rb * den);
}

__global__ void k_ds_target(DsArgs a, float tau, float* targets) {
  const int64_t nc = (int64_t)a.cx_ * a.cy_ * a.cz_;
  const int64_t X = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (X >= nc) return;
  const int x = (int)(X % a.cx_), y = (int)((X / a.cx_) % a.cy_), z = (int)(X / ((int64_t)a.cx_ * a.cy_));
  double n = 0, d = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int64_t i = cidx(a, x + dx, y + dy, z + dz);
        n += a.num[i];
        d += a.den[i];
      }
  double t = d > 0 ? -3.0 * n / d : 0.0;
  const double lo = -((double)tau - 0.5) + 1e-3;
  t = t < lo ? lo : (t > 0.5 ? 0.5 : t);
  targets[X] = (float)t;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

lbm_status lbm_closure_forward(const float* theta, const float* feats, int64_t n, int bf16,
                               float* out, void* stream) {
  set_error("");
  if (!theta || !feats || !out || n <= 0) return fail(LBM_ERR_INVALID, "bad closure_forward arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (!bf16) {
    k_mlp_forward_fp32<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(theta, feats, n, out);
    LBM_CUDA(cudaGetLastError());
    return LBM_OK;
  }
  // BF16 copy of the weights (device), as lbm_closure_load builds it
  std::vector<float> h(MLP_PARAMS);
  LBM_CUDA(cudaMemcpyAsync(h.data(), theta, MLP_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  ClosureParams cp;
  closure_params_from_fp32(h.data(), &cp);
  DevBuf d(sizeof(ClosureParams));
  if (!d.p) return fail(LBM_ERR_OOM, "device allocation failed");
  LBM_CUDA(cudaMemcpyAsync(d.p, &cp, sizeof(cp), cudaMemcpyHostToDevice, s));
  k_mlp_forward_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const ClosureParams*)d.p, feats, n, out);
  LBM_CUDA(cudaGetLastError());
  LBM_CUDA(cudaStreamSynchronize(s));
  return LBM_OK;
}

lbm_status lbm_closure_grad(const float* theta, const float* feats, const float* targets,
                            const int32_t* idx, int batch, float* grad, float* loss, void* stream) {
  set_error("");
  if (!theta || !feats || !targets || !idx || !grad || !loss || batch <= 0)
    return fail(LBM_ERR_INVALID, "bad closure_grad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<DevBuf*> keep;
  TrainBufs t;
  const bool ok = alloc_train(batch, keep, t);
  lbm_status st = LBM_OK;
  if (!ok) st = fail(LBM_ERR_OOM, "device allocation failed");
  if (!st) {
    k_gather<<<(batch + 255) / 256, 256, 0, s>>>(feats, targets, 0, idx, 0, 0, batch, nullptr, t.Xb, t.tb);
    batch_grad(theta, t, batch, grad, s);
    cudaMemcpyAsync(loss, t.loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "closure_grad");
  }
  for (auto* d : keep) delete d;
  return st;
}

lbm_status lbm_closure_train(const float* feats, const float* targets, int64_t n, int steps,
                             int batch, float lr, uint64_t seed, float* theta_io, float* loss_out,
                             void* stream) {
  set_error("");
  if (!feats || !targets || !theta_io || n <= 0 || steps <= 0 || batch <= 0)
    return fail(LBM_ERR_INVALID, "bad closure_train arguments");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<DevBuf*> keep;
  TrainBufs t;
  bool ok = alloc_train(batch, keep, t);
  DevBuf grad(MLP_PARAMS * 4), m(MLP_PARAMS * 4), v(MLP_PARAMS * 4), stats(64 * 4);
  ok = ok && grad.p && m.p && v.p && stats.p;
  lbm_status st = ok ? LBM_OK : fail(LBM_ERR_OOM, "device allocation failed");
  if (!st) {
    cudaMemsetAsync(m.p, 0, MLP_PARAMS * 4, s);
    cudaMemsetAsync(v.p, 0, MLP_PARAMS * 4, s);
    k_stats<<<MLP_IN + 1, 256, 0, s>>>(feats, targets, n, stats.f());
    for (int it = 1; it <= steps; ++it) {
      k_gather<<<(batch + 255) / 256, 256, 0, s>>>(feats, targets, n, nullptr, seed,
                                                   (int64_t)(it - 1) * batch, batch, stats.f(), t.Xb, t.tb);
      batch_grad(theta_io, t, batch, grad.f(), s);
      const float c1 = 1.f - powf(0.9f, (float)it), c2 = 1.f - powf(0.999f, (float)it);
      k_adam<<<(MLP_PARAMS + 255) / 256, 256, 0, s>>>(theta_io, grad.f(), m.f(), v.f(), MLP_PARAMS, lr, c1, c2);
    }
    if (loss_out) cudaMemcpyAsync(loss_out, t.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    // fold the normalisation into the first and last layers
    std::vector<float> th(MLP_PARAMS), sv(2 * MLP_IN + 2);
    cudaMemcpyAsync(th.data(), theta_io, MLP_PARAMS * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(sv.data(), stats.p, sv.size() * 4, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "closure_train");
    if (!st) {
      for (int j = 0; j < MLP_H; ++j) {
        double b = th[P_B1 + j];
        for (int k = 0; k < MLP_IN; ++k) {
          b -= (double)th[P_W1 + j * MLP_IN + k] * sv[k] / sv[MLP_IN + k];
          th[P_W1 + j * MLP_IN + k] /= sv[MLP_IN + k];
        }
        th[P_B1 + j] = (float)b;
        th[P_W3 + j] *= sv[2 * MLP_IN + 1];
      }
      th[P_B3] = th[P_B3] * sv[2 * MLP_IN + 1] + sv[2 * MLP_IN];
      e = cudaMemcpyAsync(theta_io, th.data(), MLP_PARAMS * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "closure_train fold");
    }
  }
  for (auto* d : keep) delete d;
  return st;
}

lbm_status lbm_closure_dataset(lbm_grid* h, int r, double tau_coarse, float* feats,
                               float* targets) {
  set_error("");
  if (!h || !feats || !targets || r < 1) return fail(LBM_ERR_INVALID, "bad closure_dataset arguments");
  Grid& g = h->g;
  if (g.kind != 0 || g.q != 19)
    return fail(LBM_ERR_UNSUPPORTED, "closure datasets come from dense D3Q19 grids");
  Level& L = g.lv[0];
  for (int a = 0; a < 3; ++a)
    if (!g.phys.periodic[a]) return fail(LBM_ERR_UNSUPPORTED, "closure datasets need a periodic box");
  if (L.nx % r || L.ny % r || L.nz % r) return fail(LBM_ERR_INVALID, "dims must be multiples of r");
  lbm_status st = lbm_sync(h);
  if (st) return st;
  DsArgs a{};
  a.f = L.f[L.cur];
  a.nx = L.nx;
  a.ny = L.ny;
  a.nz = L.nz;
  a.r = r;
  a.cx_ = L.nx / r;
  a.cy_ = L.ny / r;
  a.cz_ = L.nz / r;
  a.N = L.n_slots;
  const int64_t nc = (int64_t)a.cx_ * a.cy_ * a.cz_;
  DevBuf sbar(nc * Q * 4), mom(nc * 10 * 4), num(nc * 4), den(nc * 4);
  if (!sbar.p || !mom.p || !num.p || !den.p) return fail(LBM_ERR_OOM, "device allocation failed");
  a.sbar = sbar.f();
  a.mom = mom.f();
  a.num = num.f();
  a.den = den.f();
  cudaStream_t s = g.stream;
  const unsigned nb = (unsigned)((nc + 127) / 128);
  switch (g.phys.storage) {
    case S_F32: k_ds_filter<S_F32><<<nb, 128, 0, s>>>(a); break;
    case S_F16: k_ds_filter<S_F16><<<nb, 128, 0, s>>>(a); break;
    default: k_ds_filter<S_BF16><<<nb, 128, 0, s>>>(a); break;
  }
  k_ds_features<<<nb, 128, 0, s>>>(a, (float)tau_coarse, feats);
  k_ds_numden<<<nb, 128, 0, s>>>(a);
  k_ds_target<<<nb, 128, 0, s>>>(a, (float)tau_coarse, targets);
  LBM_CUDA(cudaGetLastError());
  LBM_CUDA(cudaStreamSynchronize(s));
  return LBM_OK;
}

lbm_status lbm_closure_load(lbm_grid* h, const float* theta, size_t n) {
  set_error("");
  if (!h || !theta) return fail(LBM_ERR_INVALID, "NULL argument");
  if (n != (size_t)MLP_PARAMS) return fail(LBM_ERR_INVALID, "closure weights must have 5313 values");
  Grid& g = h->g;
  if (g.kind != 2 || g.q != 19)
    return fail(LBM_ERR_UNSUPPORTED, "the closure runs on D3Q19 multi-resolution grids");
  ClosureParams cp;
  closure_params_from_fp32(theta, &cp);
  if (!g.closure_d) {
    g.closure_d = g.dalloc(sizeof(ClosureParams), g.stream);
    if (!g.closure_d) return fail(LBM_ERR_OOM, "device allocation failed");
  }
  LBM_CUDA(cudaMemcpyAsync(g.closure_d, &cp, sizeof(cp), cudaMemcpyHostToDevice, g.stream));
  LBM_CUDA(cudaStreamSynchronize(g.stream));
  g.closure_loaded = true;
  return LBM_OK;
}

}  // extern "C"
