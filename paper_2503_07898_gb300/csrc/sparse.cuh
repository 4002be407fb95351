// sparse.cuh - block-sparse pull of one voxel, shared by the sparse kernels,
// the multi-resolution uniform blocks and the batched persistent step
// (internal).
#pragma once
#include "d3q19.cuh"

namespace lbm {
namespace LBM_LNS {

// Pull the 19 populations of voxel l of block b (block edge E) with halfway
// bounce-back.  nbr27: the block's row of the neighbour table in global
// memory (27 ids, entry (dx+1) + 3 (dy+1) + 9 (dz+1), entry 13 = b itself,
// -1 = none); each thread reads the six entries it needs through the
// read-only cache, so a CTA starts pulling without a staging barrier.
// walls: the block or one of its 26 neighbours holds a wall voxel, or a
// neighbour is missing, so sources are checked against wm, the voxel's wall
// mask (bit i = the source of population i bounces back); a block without
// it pulls with no test at all.
//
// Address arithmetic is hoisted out of the Q pulls: a voxel can only leave
// its block across the faces it lies on, so the blocks a pull can enter —
// one per face, one per edge between two of them and, for D3Q27's corner
// velocities, the one at the corner of three (six or seven in all) — are
// looked up once, and the source coordinate wrapped into the source block
// is one of three precomputed values per axis.  Each pull then costs a few
// selects and one 32 x 32 -> 64-bit multiply-add.
template <int S, int E, bool WALLS>
__device__ __forceinline__ void sparse_pull_voxel_t(const typename Codec<S>::T* __restrict__ fin,
                                                    const int32_t* nbr27, uint32_t wm, int b,
                                                    int l, float g[Q]) {
  using T = typename Codec<S>::T;
  constexpr int E3 = E * E * E, M = E - 1;
  const int lx = l & M, ly = (l / E) & M, lz = l / (E * E);
  const int ex = lx == 0 ? -1 : (lx == M ? 1 : 0);
  const int ey = ly == 0 ? -1 : (ly == M ? 1 : 0);
  const int ez = lz == 0 ? -1 : (lz == M ? 1 : 0);
  const int nX = __ldg(nbr27 + 13 + ex), nY = __ldg(nbr27 + 13 + 3 * ey);
  const int nZ = __ldg(nbr27 + 13 + 9 * ez);
  const int nXY = __ldg(nbr27 + 13 + ex + 3 * ey), nXZ = __ldg(nbr27 + 13 + ex + 9 * ez);
  const int nYZ = __ldg(nbr27 + 13 + 3 * ey + 9 * ez);
  const int nXYZ = Q == 27 ? __ldg(nbr27 + 13 + ex + 3 * ey + 9 * ez) : b;
  // source coordinate inside its block for c = +1, -1 (pre-scaled by the
  // axis stride for y and z)
  const int xp = (lx - 1) & M, xn = (lx + 1) & M;
  const int yp = ((ly - 1) & M) * E, yn = ((ly + 1) & M) * E, y0 = ly * E;
  const int zp = ((lz - 1) & M) * E * E, zn = ((lz + 1) & M) * E * E, z0 = lz * E * E;
  const T* __restrict__ self = fin + (int64_t)b * (Q * E3) + l;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    const bool kx = X != 0 && ex == -X;  // the pull crosses the x face
    const bool ky = Y != 0 && ey == -Y;
    const bool kz = Z != 0 && ez == -Z;
    int nb = b;
    if constexpr (X != 0 && Y != 0 && Z != 0)
      nb = kz ? (kx ? (ky ? nXYZ : nXZ) : (ky ? nYZ : nZ)) : (kx ? (ky ? nXY : nX) : (ky ? nY : b));
    else if constexpr (X != 0 && Y != 0) nb = kx ? (ky ? nXY : nX) : (ky ? nY : b);
    else if constexpr (X != 0 && Z != 0) nb = kx ? (kz ? nXZ : nX) : (kz ? nZ : b);
    else if constexpr (Y != 0 && Z != 0) nb = ky ? (kz ? nYZ : nY) : (kz ? nZ : b);
    else if constexpr (X != 0) nb = kx ? nX : b;
    else if constexpr (Y != 0) nb = ky ? nY : b;
    else if constexpr (Z != 0) nb = kz ? nZ : b;
    const int ls = (X > 0 ? xp : (X < 0 ? xn : lx)) + (Y > 0 ? yp : (Y < 0 ? yn : y0)) +
                   (Z > 0 ? zp : (Z < 0 ? zn : z0));
    if constexpr (!WALLS) {
      g[I] = Codec<S>::template load<I>(fin[(int64_t)nb * (Q * E3) + (I * E3 + ls)]);
    } else {
      const bool wall = (wm >> I) & 1u;
      g[I] = Codec<S>::template load<I>(wall ? self[opp(I) * E3]
                                             : fin[(int64_t)nb * (Q * E3) + (I * E3 + ls)]);
    }
  });
}

template <int S, int E>
__device__ __forceinline__ void sparse_pull_voxel(const typename Codec<S>::T* __restrict__ fin,
                                                  const int32_t* nbr27, uint32_t wm, int64_t b,
                                                  int l, bool walls, float g[Q]) {
  if (walls) sparse_pull_voxel_t<S, E, true>(fin, nbr27, wm, (int)b, l, g);
  else sparse_pull_voxel_t<S, E, false>(fin, nbr27, 0u, (int)b, l, g);
}

}  // namespace LBM_LNS
}  // namespace lbm
