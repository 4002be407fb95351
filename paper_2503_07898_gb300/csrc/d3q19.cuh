// d3q19.cuh - D3Q19 / D3Q27 lattice, storage codecs and per-voxel update
// math (device side of liblbm).
//
// The lattice is fixed per translation unit by LBM_Q (19 by default, 27 for
// the second build of the lattice-dependent sources); everything that
// depends on it lives in namespace lbm::q19 or lbm::q27, which the rest of
// namespace lbm sees through a using-directive.  Velocity tables hold the
// 27 directions of D3Q27, whose first 19 are D3Q19 in the same order; odd i
// >= 1 has its opposite at i + 1.
//
// The paper evolves populations f_i along the D3Q19 or D3Q27 directions
// (Sec. 6 uses both lattices) by a fused
// collide-and-stream update with BGK collision (Sec. 6), halfway bounce-back
// on obstacles (Sec. 6.2) and regularized inflow / outflow boundaries
// (Sec. 6.2: they keep 3Q populations live, hence many registers).  It does
// not write the formulas; this file uses the standard forms of the
// references it cites:
//   f_i^eq   = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
//   BGK      f* = g + omega (f^eq - g),                 omega = 1 / tau
//   REG      f* = f^eq + (1 - omega) 9/2 w_i Q_i : Pi^neq
//   velocity node   rho = (S0 + 2 S+) / (1 + u_b.n)
//   pressure node   u   = ((S0 + 2 S+) / rho_b - 1) n
//   unknown c_i.n < 0: g_i = f^eq_i + g_opp(i) - f^eq_opp(i), then the
//   whole node is regularized: f* = f^eq + (1 - omega) 9/2 w_i Q_i:Pi^neq.
//
// All arithmetic runs on shifted populations s_i = f_i - w_i held in FP32
// registers: rho = 1 + sum s, j = sum c s, Pi^neq = sum c c s - (rho-1)/3 I
// - rho u u.  No O(1) constant enters an FP32 sum, so the rounding of the
// moment sums is not the same in every voxel and step (with unshifted
// values, whose low-order bits are those of the FP32 weights, that rounding
// is systematic and drifts the mass by ~3e-7 per step under 16-bit storage).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#ifndef LBM_Q
#define LBM_Q 19
#endif
#if LBM_Q == 19
#define LBM_LNS q19
#elif LBM_Q == 27
#define LBM_LNS q27
#else
#error "LBM_Q must be 19 or 27"
#endif

namespace lbm {

// Lattice tables as constexpr accessors, usable in host and device code
// (unrolled loops fold them to immediates); index < Q of the lattice in use.
__host__ __device__ constexpr int cx(int i) {
  constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0,
                         1, -1, 1, -1, 1, -1, -1, 1};
  return t[i];
}
__host__ __device__ constexpr int cy(int i) {
  constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1,
                         1, -1, 1, -1, -1, 1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz(int i) {
  constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1,
                         1, -1, -1, 1, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i & 1 ? i + 1 : i - 1); }

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

// Compile-time loop: body(integral_constant<int, I>) for I = 0..N-1.
template <int I> struct IC { static constexpr int value = I; };
template <int N, int I = 0, class F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(IC<I>{});
    static_for<N, I + 1>(f);
  }
}

enum Storage { S_F32 = 0, S_F16 = 1, S_BF16 = 2 };

namespace LBM_LNS {

constexpr int Q = LBM_Q;
// weights: D3Q19 1/3, 1/18 (axis), 1/36 (edge); D3Q27 8/27, 2/27, 1/54,
// 1/216 (corner)
__host__ __device__ constexpr double wd(int i) {
  return Q == 19 ? (i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0))
                 : (i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0)));
}
__host__ __device__ constexpr float wf(int i) { return (float)wd(i); }

// ------------------------------------------------------------ storage codecs
// F32 stores f_i.  F16 / BF16 store s_i = f_i - w_i rounded to nearest even.
// load<I> returns the shifted value s_i in FP32, store<I> takes it; abs_d
// returns the absolute f_i in FP64 (moments, reductions).

template <int S> struct Codec;
template <> struct Codec<S_F32> {
  using T = float;
  template <int I> __device__ static __forceinline__ float load(T v) { return v - wf(I); }
  template <int I> __device__ static __forceinline__ T store(float s) { return wf(I) + s; }
  __device__ static __forceinline__ float load_rt(T v, int i) { return v - wf(i); }
  __device__ static __forceinline__ double abs_d(T v, int) { return (double)v; }
  __device__ static __forceinline__ T from_double(double f, int) { return (float)f; }
};
template <> struct Codec<S_F16> {
  using T = __half;
  template <int I> __device__ static __forceinline__ float load(T v) { return __half2float(v); }
  __device__ static __forceinline__ float load_rt(T v, int) { return __half2float(v); }
  template <int I> __device__ static __forceinline__ T store(float s) { return __float2half_rn(s); }
  __device__ static __forceinline__ double abs_d(T v, int i) {
    return wd(i) + (double)__half2float(v);
  }
  __device__ static __forceinline__ T from_double(double f, int i) {
    return __double2half(f - wd(i));
  }
};
template <> struct Codec<S_BF16> {
  using T = __nv_bfloat16;
  template <int I> __device__ static __forceinline__ float load(T v) {
    return __bfloat162float(v);
  }
  __device__ static __forceinline__ float load_rt(T v, int) { return __bfloat162float(v); }
  template <int I> __device__ static __forceinline__ T store(float s) {
    return __float2bfloat16_rn(s);
  }
  __device__ static __forceinline__ double abs_d(T v, int i) {
    return wd(i) + (double)__bfloat162float(v);
  }
  __device__ static __forceinline__ T from_double(double f, int i) {
    return __double2bfloat16(f - wd(i));
  }
};

// ------------------------------------------------------------ collision
// Every function below takes and returns shifted populations s_i = f_i - w_i.

// drho = rho - 1 = sum s, j = sum c s.
// Opposite populations (i, i + 1) enter as their sum (mass) and difference
// (momentum along c_i), which saves an add per nonzero velocity component.
__device__ __forceinline__ void moments_s(const float s[Q], float& drho, float& jx, float& jy,
                                          float& jz) {
  float r = s[0], ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const float p = s[i] + s[i + 1], d = s[i] - s[i + 1];
    r += p;
    if (cx(i)) ax += cx(i) > 0 ? d : -d;
    if (cy(i)) ay += cy(i) > 0 ? d : -d;
    if (cz(i)) az += cz(i) > 0 ? d : -d;
  }
  drho = r;
  jx = ax;
  jy = ay;
  jz = az;
}

// Shifted equilibrium f^eq_i - w_i = w_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)).
__device__ __forceinline__ float eq_s(int i, float drho, float rho, float ux, float uy, float uz,
                                      float usq15) {
  const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
  return wf(i) * (drho + rho * (3.f * cu + 4.5f * cu * cu - usq15));
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

// sum_i c_ia c_ib d_i for the 6 components of a symmetric tensor.
__device__ __forceinline__ void second_moment(const float d[Q], float& sxx, float& syy, float& szz,
                                              float& sxy, float& sxz, float& syz) {
  sxx = syy = szz = sxy = sxz = syz = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (cx(i)) sxx += d[i];
    if (cy(i)) syy += d[i];
    if (cz(i)) szz += d[i];
    if (cx(i) && cy(i)) sxy += (cx(i) * cy(i) > 0) ? d[i] : -d[i];
    if (cx(i) && cz(i)) sxz += (cx(i) * cz(i) > 0) ? d[i] : -d[i];
    if (cy(i) && cz(i)) syz += (cy(i) * cz(i) > 0) ? d[i] : -d[i];
  }
}

enum Collision { C_BGK = 0, C_REG = 1 };

// In-place collision s -> s* (omega = 1 / tau).  The rest direction closes
// the mass balance: its equilibrium is drho minus the others' (the FP32
// weights sum to 1 + 1.5e-8), and for REG its non-equilibrium part is minus
// the sum of the others, so each update conserves mass up to unbiased
// rounding.
// collide_m takes the moments of s from the caller (moments_s of the same
// values), collide forms them itself.
template <int COLL>
__device__ __forceinline__ void collide_m(float s[Q], float omega, float drho, float jx, float jy,
                                          float jz) {
  const float rho = 1.f + drho;
  const float inv = 1.f / rho;
  const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  if constexpr (COLL == C_BGK) {
    // The pair (i, opp(i)) = (i, i + 1) shares the even part of the shifted
    // equilibrium: E = sym +- asym with sym = w (drho + rho (9/2 (c.u)^2 -
    // 3/2 u.u)) and asym = 3 w rho c.u, c = c_i.  The update is written
    // s* = (1 - omega) s + omega E with omega folded into the per-class
    // factors (omega w rho, omega w drho, 3 omega w rho, formed once per
    // weight class: axis, edge, corner), so each population costs one fused
    // multiply-add after its pair's omega sym +- omega asym.  The rest
    // population closes the mass: its equilibrium is drho minus twice the
    // sum of the pairs' even parts.
    constexpr float W1 = wf(1), W2 = wf(7), W3 = Q == 27 ? wf(Q - 1) : 0.f;
    constexpr float A1 = (float)(3.0 * wd(1)), A2 = (float)(3.0 * wd(7));
    constexpr float A3 = Q == 27 ? (float)(3.0 * wd(Q - 1)) : 0.f;
    const float k = 1.f - omega, orho = omega * rho, odrho = omega * drho;
    const float r1 = orho * W1, d1 = odrho * W1, a1 = orho * A1;
    const float r2 = orho * W2, d2 = odrho * W2, a2 = orho * A2;
    const float r3 = orho * W3, d3 = odrho * W3, a3 = orho * A3;
    float e = 0.f;  // sum of omega sym over the pairs
    static_for<(Q - 1) / 2>([&](auto pc) {
      constexpr int i = 2 * decltype(pc)::value + 1, o = i + 1;
      constexpr int cls = i < 7 ? 1 : (i < 19 ? 2 : 3);
      const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
      const float t = 4.5f * cu * cu - usq15;
      const float sym = cls == 1 ? fmaf(r1, t, d1) : (cls == 2 ? fmaf(r2, t, d2) : fmaf(r3, t, d3));
      const float asym = (cls == 1 ? a1 : (cls == 2 ? a2 : a3)) * cu;
      e += sym;
      s[i] = fmaf(k, s[i], sym + asym);
      s[o] = fmaf(k, s[o], sym - asym);
    });
    s[0] = fmaf(k, s[0], fmaf(-2.f, e, odrho));
  } else {
    float pxx, pyy, pzz, pxy, pxz, pyz;
    second_moment(s, pxx, pyy, pzz, pxy, pxz, pyz);
    const float d3 = drho * (1.f / 3.f);
    pxx = pxx - d3 - rho * ux * ux;
    pyy = pyy - d3 - rho * uy * uy;
    pzz = pzz - d3 - rho * uz * uz;
    pxy = pxy - rho * ux * uy;
    pxz = pxz - rho * ux * uz;
    pyz = pyz - rho * uy * uz;
    const float k = 1.f - omega;
    float e = 0.f, sn = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const float E = eq_s(i, drho, rho, ux, uy, uz, usq15);
      const float fn = reg_neq_i(i, pxx, pyy, pzz, pxy, pxz, pyz);
      e += E;
      sn += fn;
      s[i] = E + k * fn;
    }
    s[0] = (drho - e) - k * sn;
  }
}

template <int COLL>
__device__ __forceinline__ void collide(float s[Q], float omega) {
  float drho, jx, jy, jz;
  moments_s(s, drho, jx, jy, jz);
  collide_m<COLL>(s, omega, drho, jx, jy, jz);
}

// Regularized velocity / pressure node (3Q live values: s, equilibrium,
// result).  s holds the pulled populations with bounce-back already applied
// to every missing source outside the unknown set; bc = (ux, uy, uz, rho).
// With D3Q19 the weights of {c.n = 0} plus twice those of {c.n > 0} sum to
// 1, so the Zou-He density in shifted form is rho = (1 + S0 + 2 S+)/(1 + u_n).
__device__ __forceinline__ void regularized_node(float s[Q], int type, int normal, float4 bc,
                                                 float omega) {
  const int nx = normal == 0 ? 1 : (normal == 1 ? -1 : 0);
  const int ny = normal == 2 ? 1 : (normal == 3 ? -1 : 0);
  const int nz = normal == 4 ? 1 : (normal == 5 ? -1 : 0);
  float sum = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cn = cx(i) * nx + cy(i) * ny + cz(i) * nz;
    sum += cn == 0 ? s[i] : (cn > 0 ? 2.f * s[i] : 0.f);
  }
  float drho, rho, ux, uy, uz;
  if (type == T_VELOCITY) {
    ux = bc.x;
    uy = bc.y;
    uz = bc.z;
    const float un = ux * nx + uy * ny + uz * nz;
    drho = (sum - un) / (1.f + un);
    rho = 1.f + drho;
  } else {
    rho = bc.w;
    drho = bc.w - 1.f;
    const float un = (sum - drho) / rho;
    ux = un * nx;
    uy = un * ny;
    uz = un * nz;
  }
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  float E[Q];
  float e = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    E[i] = eq_s(i, drho, rho, ux, uy, uz, usq15);
    e += E[i];
  }
  E[0] = drho - e;  // mass-closing rest equilibrium (see collide)
  // non-equilibrium bounce-back of the unknown set (unknowns read known opposites)
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cn = cx(i) * nx + cy(i) * ny + cz(i) * nz;
    if (cn < 0) s[i] = E[i] + (s[opp(i)] - E[opp(i)]);
  }
  float d[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] = s[i] - E[i];
  float pxx, pyy, pzz, pxy, pxz, pyz;
  second_moment(d, pxx, pyy, pzz, pxy, pxz, pyz);
  const float k = 1.f - omega;
  float sn = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const float fn = reg_neq_i(i, pxx, pyy, pzz, pxy, pxz, pyz);
    sn += fn;
    s[i] = E[i] + k * fn;
  }
  s[0] = E[0] - k * sn;
}

// Equilibrium in FP64 (initial state, absolute).
__device__ __forceinline__ double feq_d(int i, double rho, double ux, double uy, double uz) {
  double cu = (double)cx(i) * ux + (double)cy(i) * uy + (double)cz(i) * uz;
  double usq = ux * ux + uy * uy + uz * uz;
  return wd(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

}  // namespace LBM_LNS
using namespace LBM_LNS;
}  // namespace lbm
