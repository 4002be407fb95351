// dense.cuh - dense-grid pull helpers shared by the dense kernels and the
// batched persistent step (internal).
#pragma once
#include "d3q19.cuh"
#include "grid.h"

namespace lbm {
namespace LBM_LNS {

constexpr uint32_t WM_REG = 1u << 30;   // voxel belongs to the boundary group
constexpr uint32_t WM_SKIP = 1u << 31;  // voxel not updated

struct DenseArgs {
  const void* fin;
  void* fout;
  int nx, ny, nz;
  int64_t N;
  int64_t vend;  // interior: process v < vend
  int px, py, pz;
  const uint32_t* wmask;  // null: walls only at non-periodic box sides
  const uint8_t* flags;
  const float4* bc;       // boundary: compact per list entry; monolithic: per voxel
  const int32_t* list;    // boundary voxel ids (null: contiguous from v0)
  int64_t v0, nlist;
  float omega;
};

// Pull population I of voxel (x, y, z) with halfway bounce-back.
template <int S, int I>
__device__ __forceinline__ float pull_dense(const typename Codec<S>::T* __restrict__ fin,
                                            const DenseArgs& a, int x, int y, int z, int64_t v,
                                            uint32_t wm) {
  int xs = x - cx(I), ys = y - cy(I), zs = z - cz(I);
  bool wall = false;
  if constexpr (cx(I) != 0) {
    if (xs < 0 || xs >= a.nx) {
      if (a.px) xs += xs < 0 ? a.nx : -a.nx; else wall = true;
    }
  }
  if constexpr (cy(I) != 0) {
    if (ys < 0 || ys >= a.ny) {
      if (a.py) ys += ys < 0 ? a.ny : -a.ny; else wall = true;
    }
  }
  if constexpr (cz(I) != 0) {
    if (zs < 0 || zs >= a.nz) {
      if (a.pz) zs += zs < 0 ? a.nz : -a.nz; else wall = true;
    }
  }
  if constexpr (I != 0) wall = wall || ((wm >> I) & 1u);
  const int64_t src = wall ? (int64_t)opp(I) * a.N + v
                           : (int64_t)I * a.N + xs + (int64_t)a.nx * (ys + (int64_t)a.ny * zs);
  return Codec<S>::template load<I>(fin[src]);
}

template <int S>
__device__ __forceinline__ void pull_all(const typename Codec<S>::T* __restrict__ fin,
                                         const DenseArgs& a, int x, int y, int z, int64_t v,
                                         uint32_t wm, float g[Q]) {
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    g[I] = pull_dense<S, I>(fin, a, x, y, z, v, wm);
  });
}

// Lean pull for rows without a non-periodic box side next to them in y or z
// (all rows of an axis that is periodic, the inner rows of one that is
// not): the source row offsets for c_y = +-1 and c_z = +-1 are formed once
// per voxel (wrapping across periodic sides), x edges are handled by
// predicated selects, and wall-mask bits (WM) by one bit test per
// direction.  IDX is int32_t when Q N fits in 31 bits.
template <int S, class IDX, bool WM>
__device__ __forceinline__ void pull_row_interior(const typename Codec<S>::T* __restrict__ fin,
                                                  const DenseArgs& a, int x, int y, int z, IDX v,
                                                  uint32_t wm, float g[Q]) {
  const IDX N = (IDX)a.N, nx = (IDX)a.nx, plane = (IDX)a.nx * (IDX)a.ny;
  // offset of the source row for c = +1 (row y - 1) and c = -1 (row y + 1)
  const IDX yp = y == 0 ? (IDX)(a.ny - 1) * nx : -nx;
  const IDX yn = y == a.ny - 1 ? -(IDX)(a.ny - 1) * nx : nx;
  const IDX zp = z == 0 ? (IDX)(a.nz - 1) * plane : -plane;
  const IDX zn = z == a.nz - 1 ? -(IDX)(a.nz - 1) * plane : plane;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    IDX src = (IDX)I * N + v - (IDX)cx(I);
    if constexpr (cy(I) > 0) src += yp;
    else if constexpr (cy(I) < 0) src += yn;
    if constexpr (cz(I) > 0) src += zp;
    else if constexpr (cz(I) < 0) src += zn;
    if constexpr (cx(I) > 0) {
      if (x == 0) src = a.px ? src + nx : (IDX)opp(I) * N + v;
    } else if constexpr (cx(I) < 0) {
      if (x == a.nx - 1) src = a.px ? src - nx : (IDX)opp(I) * N + v;
    }
    if constexpr (WM && I != 0) {
      if ((wm >> I) & 1u) src = (IDX)opp(I) * N + v;
    }
    g[I] = Codec<S>::template load<I>(fin[src]);
  });
}

// Lean pull of a voxel in a row with no non-periodic box side next to it in
// y or z, without per-population selects.  at(IC<I>, o) returns element
// o + c_x(I) of population I's source array, i.e. population I of voxel
// o + c_x(I); the pull source of voxel v is at(IC<I>, v + row offset of
// (c_y, c_z)), one offset per (c_y, c_z) class, wrapping across periodic
// y / z sides.  Every population is first read as if the voxel were away
// from the x ends and from walls; voxels at an x end, and voxels with
// wall-mask bits, then re-read the affected populations in branches that
// only their lanes take (bounce-back reads population opp(I) of the voxel
// itself: at(IC<opp(I)>, v - c_x(I))).  The first read of such a
// population stays inside the arrays: its element lies in [-1, N] of a
// population I >= 1 (c_x = +1 at x = 0) or I <= Q - 2 (c_x = -1 at x =
// nx - 1).  Offsets o stay within [-1, N + nx), so IDX is 32-bit while
// N + nx ny < 2^31 whatever Q N is.
template <int S, class IDX, class AT>
__device__ __forceinline__ void pull_lean(const DenseArgs& a, int x, int y, int z, IDX v,
                                          uint32_t wm, float g[Q], AT&& at) {
  const IDX nx = (IDX)a.nx, plane = (IDX)a.nx * (IDX)a.ny;
  const IDX yp = y == 0 ? (IDX)(a.ny - 1) * nx : -nx;
  const IDX yn = y == a.ny - 1 ? -(IDX)(a.ny - 1) * nx : nx;
  const IDX zp = z == 0 ? (IDX)(a.nz - 1) * plane : -plane;
  const IDX zn = z == a.nz - 1 ? -(IDX)(a.nz - 1) * plane : plane;
  auto src = [&](auto ic) -> IDX {
    constexpr int I = decltype(ic)::value;
    IDX o = v;
    if constexpr (cy(I) > 0) o += yp;
    else if constexpr (cy(I) < 0) o += yn;
    if constexpr (cz(I) > 0) o += zp;
    else if constexpr (cz(I) < 0) o += zn;
    return o;
  };
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    g[I] = Codec<S>::template load<I>(at(ic, src(ic)));
  });
  if (x == 0) {  // c_x = +1: the source lies past the row start
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if constexpr (cx(I) > 0)
        g[I] = Codec<S>::template load<I>(a.px ? at(ic, src(ic) + nx)
                                               : at(IC<opp(I)>{}, v - (IDX)cx(I)));
    });
  }
  if (x == a.nx - 1) {  // c_x = -1: the source lies past the row end
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if constexpr (cx(I) < 0)
        g[I] = Codec<S>::template load<I>(a.px ? at(ic, src(ic) - nx)
                                               : at(IC<opp(I)>{}, v - (IDX)cx(I)));
    });
  }
  if (wm) {  // sources on walls: halfway bounce-back
    static_for<Q>([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if constexpr (I != 0) {
        if ((wm >> I) & 1u) g[I] = Codec<S>::template load<I>(at(IC<opp(I)>{}, v - (IDX)cx(I)));
      }
    });
  }
}

// A row of the lean pull: no non-periodic box side next to it in y or z.
__device__ __forceinline__ bool lean_row(const DenseArgs& a, int y, int z) {
  return (a.py || (y > 0 && y < a.ny - 1)) && (a.pz || (z > 0 && z < a.nz - 1));
}

template <int S>
__device__ __forceinline__ void store_all(typename Codec<S>::T* __restrict__ fout,
                                          const DenseArgs& a, int64_t v, const float g[Q]) {
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    fout[(int64_t)I * a.N + v] = Codec<S>::template store<I>(g[I]);
  });
}

}  // namespace LBM_LNS
}  // namespace lbm
