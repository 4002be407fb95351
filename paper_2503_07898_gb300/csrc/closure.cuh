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
// mma.sync.m16n8k16 (BF16 x BF16 -> FP32) as two 16-voxel row tiles.  Each
// layer's bias enters as the MMA's accumulator input, and one
// cvt.rn.relu.bf16x2 turns two accumulators into the next layer's BF16
// operand (ReLU, round to nearest even, pack), which by the fragment layout
// of m16n8k16 is already an A fragment of the next MMA: layer 1 is 2 (M) x 8
// (N) MMAs on the 32 x 16 feature tile staged in shared memory, layer 2 is
// 2 x 8 x 4 MMAs from registers, and the output layer is an MMA against a B
// tile whose one nonzero column holds W3 (2 x 4 MMAs).  Weight fragments
// come from shared memory by ldmatrix.x4 (BF16 rows of 16-byte multiples);
// biases stay FP32.
#pragma once
#include <cuda_bf16.h>

#include "d3q19.cuh"

namespace lbm {
namespace LBM_LNS {

constexpr int MLP_IN = 16, MLP_H = 64;
constexpr int MLP_PARAMS = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;  // 5313
constexpr float TAU_MIN = 0.5f + 1e-3f;
// shared-memory row strides (BF16): 16-byte multiples (ldmatrix rows) whose
// eight rows of a fragment fall on distinct banks
constexpr int W1S = 24;
constexpr int W2S = 72;
constexpr int FSTAGE = 18;

// Device copy of a loaded network (global memory).
struct ClosureParams {
  alignas(16) __nv_bfloat16 w1[MLP_H * MLP_IN];
  alignas(16) __nv_bfloat16 w2[MLP_H * MLP_H];
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
  alignas(16) __nv_bfloat16 w1[MLP_H * W1S];
  alignas(16) __nv_bfloat16 w2[MLP_H * W2S];
  alignas(16) __nv_bfloat16 w3[MLP_H];  // BF16 (the device copy's rounded values)
  alignas(16) float b1[MLP_H];
  alignas(16) float b2[MLP_H];
  float b3;
};

// Shared memory of a 256-thread CTA running the closure: network weights and
// per-warp feature staging (dynamic, so plain kernel variants stay without it).
struct ClosureCta {
  ClosureSmem w;
  __nv_bfloat16 stage[8][32 * FSTAGE];
};

// Weights into a CTA's shared memory in 16-byte pieces (8 BF16: a W1 row is
// 2 pieces, a W2 row 8; both padded strides are 16-byte multiples).
__device__ __forceinline__ void closure_load_smem(ClosureSmem& sm, const ClosureParams* p) {
  const uint4* w1g = reinterpret_cast<const uint4*>(p->w1);
  const uint4* w2g = reinterpret_cast<const uint4*>(p->w2);
  for (int i = threadIdx.x; i < MLP_H * MLP_IN / 8; i += blockDim.x)
    *reinterpret_cast<uint4*>(sm.w1 + (i >> 1) * W1S + (i & 1) * 8) = w1g[i];
  for (int i = threadIdx.x; i < MLP_H * MLP_H / 8; i += blockDim.x)
    *reinterpret_cast<uint4*>(sm.w2 + (i >> 3) * W2S + (i & 7) * 8) = w2g[i];
  for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
    sm.w3[i] = __float2bfloat16_rn(p->w3[i]);  // exact: p->w3 holds BF16 values
    sm.b1[i] = p->b1[i];
    sm.b2[i] = p->b2[i];
  }
  if (threadIdx.x == 0) sm.b3 = p->b3;
}

// Features of one voxel from its shifted pulled populations.  The
// non-equilibrium moments are those of d = s - (f^eq - w); the equilibrium's
// own moments have closed forms (the lattice's fourth-order isotropy):
// sum c_a c_b (f^eq - w) = (rho - 1)/3 delta_ab + rho u_a u_b and
// sum c_a (|c|^2 - c_a^2) (f^eq - w) = 2/3 rho u_a (sum w c_x^2 c_y^2 = 1/9),
// so they are subtracted from the moments of s instead of forming d per
// population (equal in exact arithmetic; FP32 rounding differs).
// m receives (rho - 1, j) as moments_s gives them, for the collision.
__device__ __forceinline__ void closure_features(const float s[Q], float tau, float x[MLP_IN],
                                                 float m[4]) {
  float drho, jx, jy, jz;
  moments_s(s, drho, jx, jy, jz);
  m[0] = drho;
  m[1] = jx;
  m[2] = jy;
  m[3] = jz;
  const float rho = 1.f + drho, inv = 1.f / rho;
  const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
  float pxx, pyy, pzz, pxy, pxz, pyz;
  second_moment(s, pxx, pyy, pzz, pxy, pxz, pyz);
  const float d3 = drho * (1.f / 3.f);
  pxx -= d3 + jx * ux;
  pyy -= d3 + jy * uy;
  pzz -= d3 + jz * uz;
  pxy -= jx * uy;
  pxz -= jx * uz;
  pyz -= jy * uz;
  float qx = 0.f, qy = 0.f, qz = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int ax = cx(i), ay = cy(i), az = cz(i);
    if (ax && (ay * ay + az * az)) qx += ax > 0 ? s[i] : -s[i];
    if (ay && (ax * ax + az * az)) qy += ay > 0 ? s[i] : -s[i];
    if (az && (ax * ax + ay * ay)) qz += az > 0 ? s[i] : -s[i];
  }
  constexpr float two3 = 2.f / 3.f;
  qx -= two3 * jx;
  qy -= two3 * jy;
  qz -= two3 * jz;
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

__device__ __forceinline__ void closure_features(const float s[Q], float tau, float x[MLP_IN]) {
  float m[4];
  closure_features(s, tau, x, m);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// max(lo, 0) and max(hi, 0) rounded to BF16 (nearest even), packed with lo in
// the low half.
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// d = a * b + (c0, c1, c0, c1): the accumulator input is a per-column bias
// (columns 2q and 2q + 1 of the 16 x 8 tile).
__device__ __forceinline__ void mma_16816_bias(float d[4], const uint32_t a[4], uint32_t b0,
                                               uint32_t b1, float c0, float c1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1),
        "f"(c0), "f"(c1));
}

__device__ __forceinline__ void mma_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four 8 x 8 BF16 matrices from shared memory; lane l gives the address of
// row l % 8 of matrix l / 8 and receives, of matrix i, row l / 4 and columns
// 2 (l % 4), 2 (l % 4) + 1 in r[i].  On a weight matrix stored [unit][input]
// that is the B fragment of m16n8k16 (units n = l / 4, inputs k = 2 (l % 4)).
__device__ __forceinline__ void ldmatrix_x4(uint32_t r[4], const __nv_bfloat16* row) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((uint32_t)__cvta_generic_to_shared(row)));
}

// Network output for the calling lane's voxel; every lane of the warp must
// call it (warp-collective).  stage: this warp's 32 x FSTAGE BF16 scratch.
// The two 16-voxel row tiles run one after the other, so only one tile's
// activations are live at a time (the weight fragments are read twice).
__device__ __forceinline__ float mlp_bf16_warp(const float x[MLP_IN], const ClosureSmem& P,
                                               __nv_bfloat16* stage) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int lr = lane & 7, lm = lane >> 3;  // ldmatrix: row within, and index of, its matrix
#pragma unroll
  for (int k = 0; k < MLP_IN; k += 2)
    *reinterpret_cast<uint32_t*>(stage + lane * FSTAGE + k) = pack_bf16(x[k], x[k + 1]);
  __syncwarp();
  // column 0 of row r of a tile sits in lane 4 (r % 8), register 0 (r < 8)
  // or 2 (r >= 8); voxel (lane) L is row L % 16 of tile L / 16
  const int src = (lane & 7) * 4, my_mt = lane >> 4, my_hi = (lane >> 3) & 1;
  float out = 0.f;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    // layer 1: A = the tile's 16 x 16 features, B = W1 (64 units)
    uint32_t a1[4];
    const __nv_bfloat16* r0 = stage + (16 * mt + g) * FSTAGE;
    const __nv_bfloat16* r1 = stage + (16 * mt + g + 8) * FSTAGE;
    a1[0] = *reinterpret_cast<const uint32_t*>(r0 + 2 * q);
    a1[1] = *reinterpret_cast<const uint32_t*>(r1 + 2 * q);
    a1[2] = *reinterpret_cast<const uint32_t*>(r0 + 2 * q + 8);
    a1[3] = *reinterpret_cast<const uint32_t*>(r1 + 2 * q + 8);
    // a2[ks]: layer-2 A fragments (hidden units 16 ks .. 16 ks + 15)
    uint32_t a2[4][4];
#pragma unroll
    for (int np = 0; np < 4; ++np) {  // unit tiles 2 np and 2 np + 1
      uint32_t b[4];
      // matrices: (tile 2np, inputs 0-7), (2np, 8-15), (2np+1, 0-7), (2np+1, 8-15)
      ldmatrix_x4(b, P.w1 + (16 * np + 8 * (lm >> 1) + lr) * W1S + 8 * (lm & 1));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 bb = *reinterpret_cast<const float2*>(P.b1 + 8 * (2 * np + h) + 2 * q);
        float d[4];
        mma_16816_bias(d, a1, b[2 * h], b[2 * h + 1], bb.x, bb.y);
        a2[np][2 * h + 0] = pack_relu_bf16(d[0], d[1]);
        a2[np][2 * h + 1] = pack_relu_bf16(d[2], d[3]);
      }
    }
    // layer 2 by pairs of unit tiles; each pair completes one k-step of the
    // output layer, which runs right away (y = h2 . W3 + b3 in column 0)
    float y[4] = {P.b3, P.b3, P.b3, P.b3};
#pragma unroll 1
    for (int np = 0; np < 4; ++np) {
      uint32_t a3[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int nt = 2 * np + h;
        const float2 bb = *reinterpret_cast<const float2*>(P.b2 + 8 * nt + 2 * q);
        float acc[4];
#pragma unroll
        for (int kp = 0; kp < 2; ++kp) {  // input k-steps 2 kp and 2 kp + 1
          uint32_t b[4];
          // matrices: (k-step 2kp, half 0), (2kp, 1), (2kp+1, 0), (2kp+1, 1)
          ldmatrix_x4(b, P.w2 + (8 * nt + lr) * W2S + 32 * kp + 8 * lm);
          if (kp == 0) mma_16816_bias(acc, a2[0], b[0], b[1], bb.x, bb.y);
          else mma_16816(acc, a2[2], b[0], b[1]);
          mma_16816(acc, a2[2 * kp + 1], b[2], b[3]);
        }
        a3[2 * h + 0] = pack_relu_bf16(acc[0], acc[1]);
        a3[2 * h + 1] = pack_relu_bf16(acc[2], acc[3]);
      }
      // output layer, k-step np: B column 0 = W3[16 np .. 16 np + 15], the
      // other seven columns zero
      const uint32_t w0 = g == 0 ? *reinterpret_cast<const uint32_t*>(P.w3 + 16 * np + 2 * q) : 0u;
      const uint32_t w1 = g == 0 ? *reinterpret_cast<const uint32_t*>(P.w3 + 16 * np + 2 * q + 8) : 0u;
      mma_16816(y, a3, w0, w1);
    }
    const float v0 = __shfl_sync(0xffffffffu, y[0], src);
    const float v2 = __shfl_sync(0xffffffffu, y[2], src);
    if (my_mt == mt) out = my_hi ? v2 : v0;
  }
  __syncwarp();
  return out;
}

}  // namespace LBM_LNS
}  // namespace lbm
