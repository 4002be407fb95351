// sparse.cuh - block-sparse pull of one voxel, shared by the sparse kernels
// and the batched persistent step (internal).
#pragma once
#include "d3q19.cuh"

namespace lbm {

// Pull the 19 populations of voxel l of block b (block edge E) with halfway
// bounce-back.  nbr27: the block's 27 neighbour ids (-1 = none), usually in
// shared memory; walls: the block or its halo holds a wall voxel, so source
// flags are read; flags: per-slot flag bytes.
template <int S, int E>
__device__ __forceinline__ void sparse_pull_voxel(const typename Codec<S>::T* __restrict__ fin,
                                                  const int32_t* nbr27, const uint8_t* flags,
                                                  int64_t b, int l, bool walls, float g[Q]) {
  constexpr int E3 = E * E * E;
  const int lx = l % E, ly = (l / E) % E, lz = l / (E * E);
  static_for<Q>([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
    const int dx = sx < 0 ? -1 : (sx >= E ? 1 : 0);
    const int dy = sy < 0 ? -1 : (sy >= E ? 1 : 0);
    const int dz = sz < 0 ? -1 : (sz >= E ? 1 : 0);
    int64_t nb = b;
    if (dx | dy | dz) nb = nbr27[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
    sx -= dx * E;
    sy -= dy * E;
    sz -= dz * E;
    const int ls = sx + E * (sy + E * sz);
    bool wall = nb < 0;
    if (walls && !wall) wall = type_wall(flag_type(flags[nb * E3 + ls]));
    const int64_t src = wall ? (b * Q + opp(I)) * E3 + l : (nb * Q + I) * E3 + ls;
    g[I] = Codec<S>::template load<I>(fin[src]);
  });
}

}  // namespace lbm
