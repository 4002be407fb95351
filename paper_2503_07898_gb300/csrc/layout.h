// layout.h - sparse layout construction (classification + mapping), internal.
#pragma once
#include "grid.h"

namespace lbm {

// Classification and mapping of a block-sparse level from L.flags_h
// (virtual box) and L.E: active blocks, boundary-first (or, bitmask
// grouping, plain) Morton numbering, neighbour table, virtual block map,
// per-slot flags and wall masks (built per lattice).
namespace q19 {
lbm_status sparse_build(Grid& g, Level& L);
}
namespace q27 {
lbm_status sparse_build(Grid& g, Level& L);
}
// Upload the level's tables to the device.
lbm_status sparse_upload(Grid& g, Level& L);
// Boundary values of the regularized voxels (flag-scan order) -> boundary
// group slots.
lbm_status sparse_set_bc(Grid& g, Level& L, const float* bc_values, const float* def_bc);
// Boundary values for every slot (monolithic kernel's full-domain storage).
void sparse_fill_bc_full(const Level& L, float4* full);

uint32_t morton3(uint32_t x, uint32_t y, uint32_t z);

}  // namespace lbm
