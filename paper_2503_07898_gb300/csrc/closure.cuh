// closure.cuh - learned relaxation-time closure: features and the per-warp
// BF16 tensor-core MLP used inside the collision kernels.
//
// Not in the paper (the learned part comes from the benchmark's goal): on
// under-resolved levels of a multi-resolution grid a per-voxel network
// 16 -> 64 (ReLU) -> 64 (ReLU) -> 1 maps local moments of the pulled
// populations to a relaxation-time correction d_tau; the voxel then relaxes
// with tau_eff = max(tau + d_tau, 1/2 + 1e-3).
//
// Features (from shifted populations s = f - w; d = s - (f^eq - w)):
//   rho - 1, u, Pi^neq_{xx,yy,zz,xy,xz,yz} / (rho/3), |Pi^neq|_F / (rho/3),
//   tr Pi^neq / (rho/3), q_{x,y,z} / (rho/3) with q_x = sum c_x (c_y^2 + c_z^2) d,
//   tau.
//
// Inference: a warp evaluates the network for its 32 voxels with
// mma.sync.m16n8k16 (BF16 x BF16 -> FP32): layer 1 is 2 (M) x 8 (N) MMAs on
// the 32 x 16 feature tile staged in shared memory; its accumulators become
// the A fragments of layer 2 in registers (2 x 8 x 4 MMAs); layer 3 is a
// quad-shuffle dot product.  Weights are BF16 in shared memory, biases FP32.
#pragma once
#include <cuda_bf16.h>

#include "d3q19.cuh"

namespace lbm {
namespace LBM_LNS {

constexpr int MLP_IN = 16, MLP_H = 64;
constexpr int MLP_PARAMS = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;  // 5313
constexpr float TAU_MIN = 0.5f + 1e-3f;
constexpr int W1S = 18;  // shared-memory row strides (BF16) chosen against bank conflicts
constexpr int W2S = 72;
constexpr int FSTAGE = 18;

// Device copy of a loaded network (global memory).
struct ClosureParams {
  __nv_bfloat16 w1[MLP_H * MLP_IN];
  __nv_bfloat16 w2[MLP_H * MLP_H];
  float w3[MLP_H];  // BF16-rounded values
  float b1[MLP_H];
  float b2[MLP_H];
  float b3;
};

// Flat FP32 parameters (W1, b1, W2, b2, W3, b3) -> device layout: weights
// rounded to BF16 (nearest even), biases kept in FP32.
inline void closure_params_from_fp32(const float* th, ClosureParams* p) {
  int k = 0;
  for (int i = 0; i < MLP_H * MLP_IN; ++i) p->w1[i] = __float2bfloat16_rn(th[k++]);
  for (int i = 0; i < MLP_H; ++i) p->b1[i] = th[k++];
  for (int i = 0; i < MLP_H * MLP_H; ++i) p->w2[i] = __float2bfloat16_rn(th[k++]);
  for (int i = 0; i < MLP_H; ++i) p->b2[i] = th[k++];
  for (int i = 0; i < MLP_H; ++i) p->w3[i] = __bfloat162float(__float2bfloat16_rn(th[k++]));
  p->b3 = th[k];
}

struct ClosureSmem {
  __nv_bfloat16 w1[MLP_H * W1S];
  __nv_bfloat16 w2[MLP_H * W2S];
  float w3[MLP_H];
  float b1[MLP_H];
  float b2[MLP_H];
  float b3;
};

// Shared memory of a 256-thread CTA running the closure: network weights and
// per-warp feature staging (dynamic, so plain kernel variants stay without it).
struct ClosureCta {
  ClosureSmem w;
  __nv_bfloat16 stage[8][32 * FSTAGE];
};

__device__ __forceinline__ void closure_load_smem(ClosureSmem& sm, const ClosureParams* p) {
  for (int i = threadIdx.x; i < MLP_H * MLP_IN; i += blockDim.x)
    sm.w1[(i / MLP_IN) * W1S + i % MLP_IN] = p->w1[i];
  for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x)
    sm.w2[(i / MLP_H) * W2S + i % MLP_H] = p->w2[i];
  for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
    sm.w3[i] = p->w3[i];
    sm.b1[i] = p->b1[i];
    sm.b2[i] = p->b2[i];
  }
  if (threadIdx.x == 0) sm.b3 = p->b3;
}

// Features of one voxel from its shifted pulled populations.
__device__ __forceinline__ void closure_features(const float s[Q], float tau, float x[MLP_IN]) {
  float drho, jx, jy, jz;
  moments_s(s, drho, jx, jy, jz);
  const float rho = 1.f + drho, inv = 1.f / rho;
  const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  float d[Q];
  float e = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const float E = eq_s(i, drho, rho, ux, uy, uz, usq15);
    e += E;
    d[i] = s[i] - E;
  }
  d[0] = s[0] - (drho - e);
  float pxx, pyy, pzz, pxy, pxz, pyz;
  second_moment(d, pxx, pyy, pzz, pxy, pxz, pyz);
  float qx = 0.f, qy = 0.f, qz = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int ax = cx(i), ay = cy(i), az = cz(i);
    if (ax && (ay * ay + az * az)) qx += ax > 0 ? d[i] : -d[i];
    if (ay && (ax * ax + az * az)) qy += ay > 0 ? d[i] : -d[i];
    if (az && (ax * ax + ay * ay)) qz += az > 0 ? d[i] : -d[i];
  }
  const float k = 3.f * inv;  // 1 / (rho c_s^2)
  x[0] = drho;
  x[1] = ux;
  x[2] = uy;
  x[3] = uz;
  x[4] = pxx * k;
  x[5] = pyy * k;
  x[6] = pzz * k;
  x[7] = pxy * k;
  x[8] = pxz * k;
  x[9] = pyz * k;
  x[10] = sqrtf(x[4] * x[4] + x[5] * x[5] + x[6] * x[6] +
                2.f * (x[7] * x[7] + x[8] * x[8] + x[9] * x[9]));
  x[11] = x[4] + x[5] + x[6];
  x[12] = qx * k;
  x[13] = qy * k;
  x[14] = qz * k;
  x[15] = tau;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Network output for the calling lane's voxel; every lane of the warp must
// call it (warp-collective).  stage: this warp's 32 x FSTAGE BF16 scratch.
__device__ __forceinline__ float mlp_bf16_warp(const float x[MLP_IN], const ClosureSmem& P,
                                               __nv_bfloat16* stage) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int k = 0; k < MLP_IN; k += 2)
    *reinterpret_cast<uint32_t*>(stage + lane * FSTAGE + k) = pack_bf16(x[k], x[k + 1]);
  __syncwarp();
  uint32_t a2[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const __nv_bfloat16* r0 = stage + (16 * mt + g) * FSTAGE;
    const __nv_bfloat16* r1 = stage + (16 * mt + g + 8) * FSTAGE;
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(r0 + 2 * q);
    a[1] = *reinterpret_cast<const uint32_t*>(r1 + 2 * q);
    a[2] = *reinterpret_cast<const uint32_t*>(r0 + 2 * q + 8);
    a[3] = *reinterpret_cast<const uint32_t*>(r1 + 2 * q + 8);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int n = 8 * nt + g;
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(P.w1 + n * W1S + 2 * q);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(P.w1 + n * W1S + 2 * q + 8);
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_16816(d, a, b0, b1);
      const int c0 = 8 * nt + 2 * q;
      const float bb0 = P.b1[c0], bb1 = P.b1[c0 + 1];
      a2[mt][nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(fmaxf(d[0] + bb0, 0.f), fmaxf(d[1] + bb1, 0.f));
      a2[mt][nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(fmaxf(d[2] + bb0, 0.f), fmaxf(d[3] + bb1, 0.f));
    }
  }
  __syncwarp();
  float y[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int n = 8 * nt + g;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(P.w2 + n * W2S + 16 * ks + 2 * q);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(P.w2 + n * W2S + 16 * ks + 2 * q + 8);
      mma_16816(acc[0], a2[0][ks], b0, b1);
      mma_16816(acc[1], a2[1][ks], b0, b1);
    }
    const int c0 = 8 * nt + 2 * q;
    const float bb0 = P.b2[c0], bb1 = P.b2[c0 + 1], w0 = P.w3[c0], w1 = P.w3[c0 + 1];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      // layer-2 activations are rounded to BF16 like every layer input
      const float h0 = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[mt][0] + bb0, 0.f)));
      const float h1 = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[mt][1] + bb1, 0.f)));
      const float h2 = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[mt][2] + bb0, 0.f)));
      const float h3 = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[mt][3] + bb1, 0.f)));
      y[mt][0] += h0 * w0 + h1 * w1;
      y[mt][1] += h2 * w0 + h3 * w1;
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      y[mt][h] += __shfl_xor_sync(0xffffffffu, y[mt][h], 1);
      y[mt][h] += __shfl_xor_sync(0xffffffffu, y[mt][h], 2);
    }
  const int r = lane & 15, src = (r & 7) * 4;
  const float v00 = __shfl_sync(0xffffffffu, y[0][0], src);
  const float v01 = __shfl_sync(0xffffffffu, y[0][1], src);
  const float v10 = __shfl_sync(0xffffffffu, y[1][0], src);
  const float v11 = __shfl_sync(0xffffffffu, y[1][1], src);
  const int mtl = lane >> 4, hl = r >> 3;
  const float out = mtl == 0 ? (hl ? v01 : v00) : (hl ? v11 : v10);
  return out + P.b3;
}

}  // namespace LBM_LNS
}  // namespace lbm
