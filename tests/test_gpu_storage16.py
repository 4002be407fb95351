"""GPU: FP16 / BF16 shifted storage on the sparse and multi-resolution
layouts against the FP64 oracle.

16-bit storage rounds every stored population (f - w) once per update, so
the comparison is on the velocity field (relative L2 over the updated
voxels).  Collision damps the rounding errors of earlier steps, so the
relative velocity error stays of the order of the format's unit roundoff u
(2^-11 for FP16, 2^-8 for BF16); the bound is 4u: 2e-3 for FP16 and 1.6e-2
for BF16, after 100 updates of flows with |u| ~ 0.02-0.05.  Every boundary
kind the layouts support runs here: halfway bounce-back on a sphere and on
channel walls, regularized velocity inlet and pressure outlet, the
regularized lid of the multi-resolution cavity, and explosion / coalescence
at every level jump.
"""
import functools

import numpy as np
import pytest

from cases import bc_list, make_grid, oracle_bc, run_oracle, updated_mask
from oracle import lbm as olbm
from oracle import multires as omr
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

VEL_L2 = {"f16": 4 * 2.0 ** -11, "bf16": 4 * 2.0 ** -8}


def rel_l2(u, ur, m):
    d = (u[:, m] - ur[:, m]) ** 2
    return float(np.sqrt(d.sum() / (ur[:, m] ** 2).sum()))


def small_sphere_channel():
    return wl.sphere_channel(dims=(76, 44, 44), radius_channel=19, sphere_center_x=22,
                             sphere_radius=8, u_in=0.04)


@functools.lru_cache(maxsize=None)
def sphere_channel_oracle(collision):
    """Oracle velocity after 100 steps (independent of storage and schedule)."""
    flags, bc = small_sphere_channel()
    rho, u = wl.random_fields(flags.shape, seed=160, u_amp=0.02)
    return olbm.state_moments(run_oracle(flags, bc, rho, u, 0.56, 100, collision))[1]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("schedule,collision", [("disaggregated", "bgk"), ("bitmask", "bgk"),
                                                ("monolithic", "bgk"), ("disaggregated", "reg")])
def test_sparse_sphere_channel_16bit(lbm, storage, schedule, collision):
    """Sphere in a channel with a regularized inlet and outlet, 8^3 blocks."""
    flags, bc = small_sphere_channel()
    rho, u = wl.random_fields(flags.shape, seed=160, u_amp=0.02)
    g = make_grid(lbm, "sparse", flags, bc, 0.56, collision, storage, schedule=schedule)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, 100)
    f = lbm.lbm_get_populations_f64(g, 0)
    m = updated_mask(flags)
    assert np.all(np.isfinite(f[:, m]))
    _, u_gpu = olbm.state_moments(f)
    u_ref = sphere_channel_oracle(collision)
    err = rel_l2(u_gpu, u_ref, m)
    print(f"sparse {schedule} {collision} {storage}: velocity L2 {err:.3e}")
    assert err <= VEL_L2[storage]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_sparse_periodic_obstacles_16bit(lbm, storage):
    """Periodic box of 4^3 blocks with random obstacles (walls inside blocks
    and at block faces)."""
    shape = (32, 24, 40)
    flags = wl.random_obstacles(shape, seed=161, solid_fraction=0.1)
    rho, u = wl.random_fields(shape, seed=162, u_amp=0.02)
    g = make_grid(lbm, "sparse", flags, None, 0.6, storage=storage, periodic=(1, 1, 1),
                  block_edge=4)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, 100)
    _, u_gpu = lbm.lbm_get_moments(g, 0)
    ref = run_oracle(flags, None, rho, u, 0.6, 100, periodic=(1, 1, 1))
    _, u_ref = olbm.state_moments(ref)
    err = rel_l2(u_gpu, u_ref, updated_mask(flags))
    print(f"sparse periodic obstacles {storage}: velocity L2 {err:.3e}")
    assert err <= VEL_L2[storage]


# ------------------------------------------------------------------ dense
# The 16-bit dense interior kernel reads every population as if the voxel
# were away from the x ends and from walls and re-reads the affected ones
# for voxels at an x end or next to a wall; these cases take every such
# branch: x ends that wrap and x ends that bounce back, a per-voxel wall
# mask (obstacles, regularized inlet / outlet), y / z box sides of both kinds.

@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_dense_channel_obstacles_16bit(lbm, storage):
    """Obstacles, regularized inlet / outlet, bounce-back side walls (x, y,
    z not periodic): the wall-mask path."""
    dims_zyx = (14, 18, 41)
    flags = wl.random_obstacles(dims_zyx, seed=24, solid_fraction=0.08)
    flags[:, :, 0] = wl.flag(wl.VELOCITY, wl.NX_M)
    flags[:, :, -1] = wl.flag(wl.PRESSURE, wl.NX_P)
    bc = np.zeros((4,) + dims_zyx)
    bc[0, :, :, 0] = 0.03
    bc[3] = 1.0
    bc[3, :, :, -1] = 0.995
    rho, u = wl.random_fields(dims_zyx, seed=25, u_amp=0.02)
    g = make_grid(lbm, "dense", flags, bc, 0.58, storage=storage)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, 100)
    f = lbm.lbm_get_populations_f64(g, 0)
    m = updated_mask(flags)
    assert np.all(np.isfinite(f[:, m]))
    _, u_gpu = olbm.state_moments(f)
    _, u_ref = olbm.state_moments(run_oracle(flags, bc, rho, u, 0.58, 100))
    err = rel_l2(u_gpu, u_ref, m)
    print(f"dense channel obstacles {storage}: velocity L2 {err:.3e}")
    assert err <= VEL_L2[storage]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("periodic", [(1, 0, 1), (0, 1, 1)])
def test_dense_obstacles_mixed_periodic_16bit(lbm, storage, periodic):
    """Obstacles on a box periodic along some axes: x ends that wrap or
    bounce back, with the wall mask, on a ragged 37 x 19 x 23 box."""
    dims_zyx = (23, 19, 37)
    flags = wl.random_obstacles(dims_zyx, seed=26, solid_fraction=0.06)
    rho, u = wl.random_fields(dims_zyx, seed=27, u_amp=0.03)
    g = make_grid(lbm, "dense", flags, None, 0.6, storage=storage, periodic=periodic)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, 100)
    f = lbm.lbm_get_populations_f64(g, 0)
    m = updated_mask(flags)
    assert np.all(np.isfinite(f[:, m]))
    _, u_gpu = olbm.state_moments(f)
    _, u_ref = olbm.state_moments(run_oracle(flags, None, rho, u, 0.6, 100,
                                             periodic=periodic))
    err = rel_l2(u_gpu, u_ref, m)
    print(f"dense obstacles periodic {periodic} {storage}: velocity L2 {err:.3e}")
    assert err <= VEL_L2[storage]


def channel_flags(dims_zyx, seed):
    """A channel along x (circular cross-section, not-in-domain voxels
    outside it, so whole blocks are missing and partly filled blocks hold
    masked voxels) with random solids inside."""
    nz, ny, nx = dims_zyx
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    inside = np.broadcast_to((y - ny / 2 + 0.5) ** 2 + (z - nz / 2 + 0.5) ** 2 < (0.45 * nz) ** 2,
                             dims_zyx)
    flags = wl.random_obstacles(dims_zyx, seed=seed, solid_fraction=0.05)
    flags[~inside] = wl.OUTSIDE
    return flags


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("collision", ["bgk", "reg"])
@pytest.mark.parametrize("layout", ["periodic", "obstacle", "channel"])
def test_sparse_16bit_equals_dense_16bit(lbm, storage, collision, layout):
    """The block-sparse 16-bit step (two voxels per thread; in blocks with
    walls, the warps whose z plane holds a wall bit update one voxel at a
    time and the others keep the two-voxel form) gives the dense 16-bit
    step's populations bit for bit: both pull the same stored values and run
    the same collision.  Layouts: a periodic box with every block active,
    the same with a solid box, and a channel periodic along x only (missing
    blocks outside it, not-in-domain and solid voxels inside blocks,
    bounce-back at the y / z box sides)."""
    dims_zyx = (24, 32, 48)
    periodic = (1, 1, 1)
    flags = np.zeros(dims_zyx, np.uint8)
    if layout == "obstacle":
        flags[3:9, 10:15, 30:37] = wl.SOLID
    elif layout == "channel":
        dims_zyx = (32, 40, 48)
        flags = channel_flags(dims_zyx, seed=29)
        periodic = (1, 0, 0)
    rho, u = wl.random_fields(dims_zyx, seed=28, u_amp=0.03)
    out = []
    for kind in ("dense", "sparse"):
        g = make_grid(lbm, kind, flags, None, 0.57, collision, storage, periodic=periodic)
        lbm.lbm_init_equilibrium(g, 0, rho, u)
        lbm.lbm_step(g, 40)
        out.append(lbm.lbm_get_populations_f64(g, 0))
    m = updated_mask(flags)
    assert np.all(np.isfinite(out[0][:, m]))
    assert np.array_equal(out[0][:, m], out[1][:, m])


# ------------------------------------------------------- multi-resolution

LMAP3 = np.array([2, 1, 0, 1], np.uint8).reshape(4, 1, 1)


def level_init(dims, n_levels, seed):
    out = []
    for lv in range(n_levels):
        nx, ny, nz = (d >> lv for d in dims)
        out.append(wl.random_fields((nz, ny, nx), seed=seed + lv, u_amp=0.02))
    return out


@functools.lru_cache(maxsize=None)
def three_level_oracle():
    """Oracle after 25 coarsest steps (independent of storage and schedule)."""
    o = omr.MultiRes(LMAP3, 3, 32, 0.58)
    for lv, (rho, u) in enumerate(level_init((32, 32, 128), 3, 163)):
        o.init_equilibrium(lv, rho, u)
    o.run(25)
    return o


def mr_velocity_errors(lbm, g, o, n_levels):
    """Relative velocity L2 of each level over the voxels that level owns."""
    out = []
    for lv in range(n_levels):
        m = o.own[lv] == lv
        if not m.any():
            continue
        f = lbm.lbm_get_populations_f64(g, lv)
        assert np.all(np.isfinite(f[:, m]))
        _, u_gpu = olbm.state_moments(f)
        _, u_ref = olbm.state_moments(o.f[lv])
        out.append(rel_l2(u_gpu, u_ref, m))
    return out


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("schedule", ["disaggregated", "monolithic"])
def test_multires_three_level_16bit(lbm, storage, schedule):
    """Periodic three-level map with every jump of the turbulence workload
    (coarse - middle - fine - middle), 25 coarsest steps = 100 finest
    updates."""
    cell = 32
    dims = (cell, cell, 4 * cell)
    g = lbm.lbm_grid_create_multires(dims, 3, LMAP3, lbm.physics(
        0.58, "bgk", storage, (1, 1, 1), schedule))
    for lv, (rho, u) in enumerate(level_init(dims, 3, 163)):
        lbm.lbm_init_equilibrium(g, lv, rho, u)
    lbm.lbm_step(g, 25)
    o = three_level_oracle()
    errs = mr_velocity_errors(lbm, g, o, 3)
    print(f"multires {schedule} {storage}: velocity L2 per level {errs}")
    assert max(errs) <= VEL_L2[storage]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_multires_cavity_16bit(lbm, storage):
    """Two-level lid-driven cavity (walls and regularized lid on level 0), 50
    coarsest steps."""
    n = 48
    lmap = wl.multires_cavity_map(n, 2, (1,))
    g = lbm.lbm_grid_create_multires((n,) * 3, 2, lmap, lbm.physics(
        0.6, "bgk", storage, (0, 0, 0)))
    flags, bc = wl.cavity(n)
    lbm.lbm_set_boundary(g, 0, flags, bc_list(flags, bc))
    o = omr.MultiRes(lmap, 2, 16, 0.6, periodic=(False,) * 3, flags0=flags,
                     bc0=oracle_bc(flags, bc))
    rho, u = wl.random_fields((n,) * 3, seed=166, u_amp=0.02)
    fields = [(rho, u), (omr.subcell_mean(rho), omr.subcell_mean(u))]
    for lv, (r, v) in enumerate(fields):
        lbm.lbm_init_equilibrium(g, lv, r, v)
        o.init_equilibrium(lv, r, v)
    lbm.lbm_step(g, 50)               # 100 level-0 substeps
    o.run(50)
    errs = mr_velocity_errors(lbm, g, o, 2)
    print(f"multires cavity {storage}: velocity L2 per level {errs}")
    assert max(errs) <= VEL_L2[storage]
