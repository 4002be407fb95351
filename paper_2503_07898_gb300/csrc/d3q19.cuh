// d3q19.cuh - D3Q19 lattice, storage codecs and per-voxel update math
// (device side of liblbm).
//
// The paper evolves populations f_i along the D3Q19 directions by a fused
// collide-and-stream update with BGK collision (Sec. 6), halfway bounce-back
// on obstacles (Sec. 6.2) and regularized inflow / outflow boundaries
// (Sec. 6.2, "register-heavy", 3Q live populations).  It does not write the
// formulas; this file uses the standard forms of the references it cites:
//   f_i^eq   = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
//   BGK      f* = g + omega (f^eq - g),                 omega = 1 / tau
//   REG      f* = f^eq + (1 - omega) 9/2 w_i Q_i : Pi^neq
//   velocity node   rho = (S0 + 2 S+) / (1 + u_b.n)
//   pressure node   u   = ((S0 + 2 S+) / rho_b - 1) n
//   unknown c_i.n < 0: g_i = f^eq_i + g_opp(i) - f^eq_opp(i), then the
//   whole node is regularized: f* = f^eq + (1 - omega) 9/2 w_i Q_i:Pi^neq.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbm {

constexpr int Q = 19;
// Lattice tables as constexpr accessors, usable in host and device code
// (unrolled loops fold them to immediates).
__host__ __device__ constexpr int cx(int i) {
  constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return t[i];
}
__host__ __device__ constexpr int opp(int i) {
  constexpr int t[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
  return t[i];
}
__host__ __device__ constexpr float wf(int i) {
  return i == 0 ? 1.f / 3.f : (i <= 6 ? 1.f / 18.f : 1.f / 36.f);
}
__host__ __device__ constexpr double wd(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Flag byte.
constexpr int T_FLUID = 0, T_SOLID = 1, T_VELOCITY = 2, T_PRESSURE = 3, T_OUTSIDE = 7;
__host__ __device__ inline int flag_type(uint8_t f) { return f & 7; }
__host__ __device__ inline int flag_normal(uint8_t f) { return (f >> 3) & 7; }
__host__ __device__ inline bool type_updated(int t) {
  return t == T_FLUID || t == T_VELOCITY || t == T_PRESSURE;
}
__host__ __device__ inline bool type_wall(int t) { return t == T_SOLID || t == T_OUTSIDE; }
__host__ __device__ inline bool type_regularized(int t) {
  return t == T_VELOCITY || t == T_PRESSURE;
}

// ------------------------------------------------------------ storage codecs
// F32 stores f_i.  F16 / BF16 store s_i = f_i - w_i rounded to nearest even;
// a load returns w_i + s_i in FP32.
enum Storage { S_F32 = 0, S_F16 = 1, S_BF16 = 2 };

template <int S> struct Codec;
template <> struct Codec<S_F32> {
  using T = float;
  template <int I> __device__ static __forceinline__ float load(T v) { return v; }
  template <int I> __device__ static __forceinline__ T store(float f) { return f; }
  __device__ static __forceinline__ float load_i(T v, int) { return v; }
  __device__ static __forceinline__ T from_double(double f, int) { return (float)f; }
};
template <> struct Codec<S_F16> {
  using T = __half;
  template <int I> __device__ static __forceinline__ float load(T v) {
    return wf(I) + __half2float(v);
  }
  template <int I> __device__ static __forceinline__ T store(float f) {
    return __float2half_rn(f - wf(I));
  }
  __device__ static __forceinline__ float load_i(T v, int i) { return wf(i) + __half2float(v); }
  __device__ static __forceinline__ T from_double(double f, int i) {
    return __double2half(f - wd(i));
  }
};
template <> struct Codec<S_BF16> {
  using T = __nv_bfloat16;
  template <int I> __device__ static __forceinline__ float load(T v) {
    return wf(I) + __bfloat162float(v);
  }
  template <int I> __device__ static __forceinline__ T store(float f) {
    return __float2bfloat16_rn(f - wf(I));
  }
  __device__ static __forceinline__ float load_i(T v, int i) {
    return wf(i) + __bfloat162float(v);
  }
  __device__ static __forceinline__ T from_double(double f, int i) {
    return __double2bfloat16(f - wd(i));
  }
};

// Compile-time loop: body(integral_constant<int, I>) for I = 0..N-1.
template <int I> struct IC { static constexpr int value = I; };
template <int N, int I = 0, class F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(IC<I>{});
    static_for<N, I + 1>(f);
  }
}

// ------------------------------------------------------------ collision

// Moments of a population set.
__device__ __forceinline__ void moments(const float g[Q], float& rho, float& ux, float& uy,
                                        float& uz) {
  float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    r += g[i];
    if (cx(i)) jx += cx(i) > 0 ? g[i] : -g[i];
    if (cy(i)) jy += cy(i) > 0 ? g[i] : -g[i];
    if (cz(i)) jz += cz(i) > 0 ? g[i] : -g[i];
  }
  float inv = 1.f / r;
  rho = r;
  ux = jx * inv;
  uy = jy * inv;
  uz = jz * inv;
}

__device__ __forceinline__ float feq_i(int i, float rho, float ux, float uy, float uz,
                                       float usq15) {
  float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
  return wf(i) * rho * (1.f + 3.f * cu + 4.5f * cu * cu - usq15);
}

// 9/2 w_i Q_i : P for a symmetric tensor P given by its 6 components.
__device__ __forceinline__ float reg_neq_i(int i, float pxx, float pyy, float pzz, float pxy,
                                           float pxz, float pyz) {
  const float ex = (float)cx(i), ey = (float)cy(i), ez = (float)cz(i);
  const float third = 1.f / 3.f;
  float q = (ex * ex - third) * pxx + (ey * ey - third) * pyy + (ez * ez - third) * pzz +
            2.f * (ex * ey * pxy + ex * ez * pxz + ey * ez * pyz);
  return 4.5f * wf(i) * q;
}

// Non-equilibrium second moment Pi^neq = sum c c g - rho (I/3 + u u).
__device__ __forceinline__ void pi_neq(const float g[Q], float rho, float ux, float uy, float uz,
                                       float& pxx, float& pyy, float& pzz, float& pxy,
                                       float& pxz, float& pyz) {
  float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (cx(i)) sxx += g[i];
    if (cy(i)) syy += g[i];
    if (cz(i)) szz += g[i];
    if (cx(i) && cy(i)) sxy += (cx(i) * cy(i) > 0) ? g[i] : -g[i];
    if (cx(i) && cz(i)) sxz += (cx(i) * cz(i) > 0) ? g[i] : -g[i];
    if (cy(i) && cz(i)) syz += (cy(i) * cz(i) > 0) ? g[i] : -g[i];
  }
  const float r3 = rho * (1.f / 3.f);
  pxx = sxx - r3 - rho * ux * ux;
  pyy = syy - r3 - rho * uy * uy;
  pzz = szz - r3 - rho * uz * uz;
  pxy = sxy - rho * ux * uy;
  pxz = sxz - rho * ux * uz;
  pyz = syz - rho * uy * uz;
}

enum Collision { C_BGK = 0, C_REG = 1 };

// In-place collision of pulled populations g -> f*.  omega = 1 / tau.
//
// The FP32-rounded weights sum to 1 + 1.5e-8, which would add a systematic
// omega * 1.5e-8 * rho of mass per voxel and step.  The rest direction
// therefore closes the balance: f^eq_0 = rho - sum_{i>0} f^eq_i (and the
// regularized non-equilibrium part of i = 0 is minus the sum of the others),
// so each update conserves mass up to unbiased rounding.
template <int COLL>
__device__ __forceinline__ void collide(float g[Q], float omega) {
  float rho, ux, uy, uz;
  moments(g, rho, ux, uy, uz);
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  if constexpr (COLL == C_BGK) {
    float s = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const float fe = feq_i(i, rho, ux, uy, uz, usq15);
      s += fe;
      g[i] = g[i] + omega * (fe - g[i]);
    }
    g[0] = g[0] + omega * ((rho - s) - g[0]);
  } else {
    float pxx, pyy, pzz, pxy, pxz, pyz;
    pi_neq(g, rho, ux, uy, uz, pxx, pyy, pzz, pxy, pxz, pyz);
    const float k = 1.f - omega;
    float s = 0.f, sn = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const float fe = feq_i(i, rho, ux, uy, uz, usq15);
      const float fn = reg_neq_i(i, pxx, pyy, pzz, pxy, pxz, pyz);
      s += fe;
      sn += fn;
      g[i] = fe + k * fn;
    }
    g[0] = (rho - s) - k * sn;
  }
}

// Regularized velocity / pressure node (3Q live values: g, f^eq, result).
// g holds the pulled populations with bounce-back already applied to every
// missing source outside the unknown set; bc = (ux, uy, uz, rho).
__device__ __forceinline__ void regularized_node(float g[Q], int type, int normal, float4 bc,
                                                 float omega) {
  const int nx = normal == 0 ? 1 : (normal == 1 ? -1 : 0);
  const int ny = normal == 2 ? 1 : (normal == 3 ? -1 : 0);
  const int nz = normal == 4 ? 1 : (normal == 5 ? -1 : 0);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cn = cx(i) * nx + cy(i) * ny + cz(i) * nz;
    s += cn == 0 ? g[i] : (cn > 0 ? 2.f * g[i] : 0.f);
  }
  float rho, ux, uy, uz;
  if (type == T_VELOCITY) {
    ux = bc.x;
    uy = bc.y;
    uz = bc.z;
    rho = s / (1.f + (ux * nx + uy * ny + uz * nz));
  } else {
    rho = bc.w;
    const float un = s / rho - 1.f;
    ux = un * nx;
    uy = un * ny;
    uz = un * nz;
  }
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  float feq[Q];
  float s_eq = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    feq[i] = feq_i(i, rho, ux, uy, uz, usq15);
    s_eq += feq[i];
  }
  feq[0] = rho - s_eq;  // mass-closing rest equilibrium (see collide)
  // non-equilibrium bounce-back of the unknown set (unknowns read known opposites)
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cn = cx(i) * nx + cy(i) * ny + cz(i) * nz;
    if (cn < 0) g[i] = feq[i] + (g[opp(i)] - feq[opp(i)]);
  }
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const float d = g[i] - feq[i];
    if (cx(i)) pxx += d;
    if (cy(i)) pyy += d;
    if (cz(i)) pzz += d;
    if (cx(i) && cy(i)) pxy += (cx(i) * cy(i) > 0) ? d : -d;
    if (cx(i) && cz(i)) pxz += (cx(i) * cz(i) > 0) ? d : -d;
    if (cy(i) && cz(i)) pyz += (cy(i) * cz(i) > 0) ? d : -d;
  }
  // the rest population enters Pi only through the trace-free projection: c_0 = 0
  const float k = 1.f - omega;
  float s_neq = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const float fn = reg_neq_i(i, pxx, pyy, pzz, pxy, pxz, pyz);
    s_neq += fn;
    g[i] = feq[i] + k * fn;
  }
  g[0] = feq[0] - k * s_neq;
}

// Equilibrium in FP64 (initial state).
__device__ __forceinline__ double feq_d(int i, double rho, double ux, double uy, double uz) {
  double cu = (double)cx(i) * ux + (double)cy(i) * uy + (double)cz(i) * uz;
  double usq = ux * ux + uy * uy + uz * uz;
  return wd(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

}  // namespace lbm
