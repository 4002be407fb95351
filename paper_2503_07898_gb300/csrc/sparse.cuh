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
// selects among the neighbours' element offsets (formed once per voxel), one
// add and the load.  IDX is int32_t when the level's Q E^3 n_blocks elements
// fit in 31 bits (the kernels choose), else int64_t.
template <int S, int E, bool WALLS, class IDX = int64_t>
__device__ __forceinline__ void sparse_pull_voxel_t(const typename Codec<S>::T* __restrict__ fin,
                                                    const int32_t* nbr27, uint32_t wm, int b,
                                                    int l, float g[Q]) {
  using T = typename Codec<S>::T;
  constexpr int E3 = E * E * E, M = E - 1;
  constexpr IDX QE3 = (IDX)Q * E3;
  const int lx = l & M, ly = (l / E) & M, lz = l / (E * E);
  const int ex = lx == 0 ? -1 : (lx == M ? 1 : 0);
  const int ey = ly == 0 ? -1 : (ly == M ? 1 : 0);
  const int ez = lz == 0 ? -1 : (lz == M ? 1 : 0);
  // element offsets of the blocks a pull can enter (a missing neighbour
  // gives a negative offset that only a bounced-back pull would name, and
  // such a pull reads the voxel itself instead)
  const IDX oS = (IDX)b * QE3;
  const IDX oX = (IDX)__ldg(nbr27 + 13 + ex) * QE3, oY = (IDX)__ldg(nbr27 + 13 + 3 * ey) * QE3;
  const IDX oZ = (IDX)__ldg(nbr27 + 13 + 9 * ez) * QE3;
  const IDX oXY = (IDX)__ldg(nbr27 + 13 + ex + 3 * ey) * QE3;
  const IDX oXZ = (IDX)__ldg(nbr27 + 13 + ex + 9 * ez) * QE3;
  const IDX oYZ = (IDX)__ldg(nbr27 + 13 + 3 * ey + 9 * ez) * QE3;
  const IDX oXYZ = Q == 27 ? (IDX)__ldg(nbr27 + 13 + ex + 3 * ey + 9 * ez) * QE3 : oS;
  // source coordinate inside its block for c = +1, -1 (pre-scaled by the
  // axis stride for y and z)
  const int xp = (lx - 1) & M, xn = (lx + 1) & M;
  const int yp = ((ly - 1) & M) * E, yn = ((ly + 1) & M) * E, y0 = ly * E;
  const int zp = ((lz - 1) & M) * E * E, zn = ((lz + 1) & M) * E * E, z0 = lz * E * E;
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    const bool kx = X != 0 && ex == -X;  // the pull crosses the x face
    const bool ky = Y != 0 && ey == -Y;
    const bool kz = Z != 0 && ez == -Z;
    IDX o = oS;
    if constexpr (X != 0 && Y != 0 && Z != 0)
      o = kz ? (kx ? (ky ? oXYZ : oXZ) : (ky ? oYZ : oZ)) : (kx ? (ky ? oXY : oX) : (ky ? oY : oS));
    else if constexpr (X != 0 && Y != 0) o = kx ? (ky ? oXY : oX) : (ky ? oY : oS);
    else if constexpr (X != 0 && Z != 0) o = kx ? (kz ? oXZ : oX) : (kz ? oZ : oS);
    else if constexpr (Y != 0 && Z != 0) o = ky ? (kz ? oYZ : oY) : (kz ? oZ : oS);
    else if constexpr (X != 0) o = kx ? oX : oS;
    else if constexpr (Y != 0) o = ky ? oY : oS;
    else if constexpr (Z != 0) o = kz ? oZ : oS;
    const int ls = (X > 0 ? xp : (X < 0 ? xn : lx)) + (Y > 0 ? yp : (Y < 0 ? yn : y0)) +
                   (Z > 0 ? zp : (Z < 0 ? zn : z0));
    IDX src = o + (IDX)(I * E3 + ls);
    if constexpr (WALLS) {
      if ((wm >> I) & 1u) src = oS + (IDX)(opp(I) * E3 + l);
    }
    g[I] = Codec<S>::template load<I>(fin[src]);
  });
}

template <int S, int E, class IDX = int64_t>
__device__ __forceinline__ void sparse_pull_voxel(const typename Codec<S>::T* __restrict__ fin,
                                                  const int32_t* nbr27, uint32_t wm, int64_t b,
                                                  int l, bool walls, float g[Q]) {
  if (walls) sparse_pull_voxel_t<S, E, true, IDX>(fin, nbr27, wm, (int)b, l, g);
  else sparse_pull_voxel_t<S, E, false, IDX>(fin, nbr27, 0u, (int)b, l, g);
}

}  // namespace LBM_LNS
}  // namespace lbm
