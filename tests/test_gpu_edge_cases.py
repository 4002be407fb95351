"""GPU: degenerate inputs against the oracle or their exact outcome.

Single-voxel and one-voxel-thick boxes (every pull wraps onto the voxel
itself or bounces back), grids with no updated voxel at all, a sparse grid
with a single active block, and a multi-resolution grid whose coarsest level
owns nothing.
"""
import numpy as np
import pytest

from cases import F32_RTOL, make_grid, max_rel_err, run_oracle
from oracle import multires as omr
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def gpu_run(lbm, g, rho, u, steps):
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, steps)
    return lbm.lbm_get_populations_f64(g, 0)


@pytest.mark.parametrize("dims_zyx,periodic", [
    ((1, 1, 1), (1, 1, 1)),
    ((5, 7, 1), (1, 0, 1)),
    ((4, 1, 9), (0, 1, 0)),
    ((1, 5, 6), (0, 0, 1)),
    ((12, 1, 1), (0, 0, 0)),
])
@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_tiny_and_one_voxel_thick_boxes(lbm, dims_zyx, periodic, kind):
    flags = np.zeros(dims_zyx, np.uint8)
    if kind == "sparse" and any(p and n % 4 for p, n in zip(periodic, dims_zyx[::-1])):
        # a periodic axis of a block-sparse grid must hold whole blocks: the
        # library refuses the grid instead of wrapping inside a block
        with pytest.raises(lbm.LbmError) as e:
            make_grid(lbm, kind, flags, None, 0.6, periodic=periodic, block_edge=4)
        assert e.value.status == lbm.LBM_ERR_INVALID
        assert "divisible by block_edge" in str(e.value)
        return
    rho, u = wl.random_fields(dims_zyx, seed=150, u_amp=0.02)
    g = make_grid(lbm, kind, flags, None, 0.6, periodic=periodic, block_edge=4)
    f = gpu_run(lbm, g, rho, u, 30)
    ref = run_oracle(flags, None, rho, u, 0.6, 30, periodic=periodic)
    assert max_rel_err(f, ref, flags) <= F32_RTOL


@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_grid_without_updated_voxels(lbm, kind):
    """Every voxel solid: stepping is a no-op, populations decode to NaN and
    the conservation sums are zero."""
    flags = np.full((8, 9, 10), wl.SOLID, np.uint8)
    g = make_grid(lbm, kind, flags, None, 0.6)
    info = lbm.lbm_get_info(g)
    assert info["n_updated"][0] == 0
    lbm.lbm_init_equilibrium(g, 0, None, None)
    lbm.lbm_step(g, 3)
    assert np.all(np.isnan(lbm.lbm_get_populations_f64(g, 0)))
    assert np.all(lbm.lbm_conservation(g) == 0.0)


def test_sparse_single_active_block(lbm):
    flags = np.full((24, 24, 24), wl.OUTSIDE, np.uint8)
    flags[8:16, 8:16, 8:16] = wl.FLUID
    flags[10, 12, 11] = wl.SOLID
    rho, u = wl.random_fields(flags.shape, seed=151, u_amp=0.02)
    g = make_grid(lbm, "sparse", flags, None, 0.58)
    assert lbm.lbm_get_info(g)["n_blocks"][0] == 1
    f = gpu_run(lbm, g, rho, u, 40)
    ref = run_oracle(flags, None, rho, u, 0.58, 40)
    assert max_rel_err(f, ref, flags) <= F32_RTOL


def test_multires_level_without_blocks(lbm):
    """A 3-level grid whose map uses levels 0 and 1 only: level 2 stays
    empty (NaN everywhere), the others match the oracle."""
    lmap = np.array([1, 0, 0, 1], np.uint8).reshape(4, 1, 1)
    dims = (32, 32, 128)
    g = lbm.lbm_grid_create_multires(dims, 3, lmap, lbm.physics(0.6, periodic=(1, 1, 1)))
    o = omr.MultiRes(lmap, 3, 32, 0.6)
    for lv in range(3):
        nx, ny, nz = (d >> lv for d in dims)
        rho, u = wl.random_fields((nz, ny, nx), seed=152 + lv, u_amp=0.02)
        lbm.lbm_init_equilibrium(g, lv, rho, u)
        o.init_equilibrium(lv, rho, u)
    assert lbm.lbm_get_info(g)["n_blocks"][2] == 0
    lbm.lbm_step(g, 2)
    o.run(2)
    for lv in range(2):
        f = lbm.lbm_get_populations_f64(g, lv)
        m = o.own[lv] == lv
        ref = o.f[lv][:, m]
        assert np.max(np.abs(f[:, m] - ref) / np.abs(ref)) <= F32_RTOL
    assert np.all(np.isnan(lbm.lbm_get_populations_f64(g, 2)))


@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_non_finite_state_is_reported_as_diverged(lbm, kind):
    """A non-finite population (planted through the checkpoint path, on the
    host) spreads through the pull and collision; the conservation sums then
    report LBM_ERR_DIVERGED instead of returning NaN."""
    flags = np.zeros((16, 16, 16), np.uint8)
    g = make_grid(lbm, kind, flags, None, 0.6, periodic=(1, 1, 1))
    rho, u = wl.random_fields(flags.shape, seed=153, u_amp=0.02)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    assert np.all(np.isfinite(lbm.lbm_conservation(g)))
    f = np.empty(19 * 16 ** 3, np.float32)
    lbm.lbm_get_populations(g, 0, f)
    f[5 * 16 ** 3 + 100] = np.nan
    lbm.lbm_set_populations(g, 0, f)
    lbm.lbm_step(g, 3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_conservation(g)
    assert "DIVERGED" in str(e.value)
