"""GPU: multi-resolution grids against the FP64 multi-resolution oracle.

Parity cases use level maps with every level jump of the 3-level turbulence
workload (coarse - middle - fine - middle along z) at the smallest sizes the
8^3-block layout allows; the full 256^3 three-level workload is checked by
properties that hold at any size (exact volume-weighted conservation up to
FP32 rounding, fused == unfused bit for bit, voxel counts).
"""
import numpy as np
import pytest

from cases import F32_RTOL, bc_list, oracle_bc
from oracle import layout as olayout
from oracle import multires as omr
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def make_mr(lbm, lmap, n_levels, tau, schedule="disaggregated", storage="f32", collision="bgk"):
    cell = 8 * 2 ** (n_levels - 1)
    mz, my, mx = lmap.shape
    dims = (mx * cell, my * cell, mz * cell)
    g = lbm.lbm_grid_create_multires(dims, n_levels, lmap, lbm.physics(
        tau, collision, storage, (1, 1, 1), schedule))
    return g, dims, cell


def level_fields(dims, n_levels, seed):
    out = []
    for lv in range(n_levels):
        nx, ny, nz = (d >> lv for d in dims)
        out.append(wl.random_fields((nz, ny, nx), seed=seed + lv, u_amp=0.02))
    return out


def init_both(lbm, g, o, fields):
    for lv, (rho, u) in enumerate(fields):
        lbm.lbm_init_equilibrium(g, lv, rho, u)
        o.init_equilibrium(lv, rho, u)


def compare(lbm, g, o, n_levels):
    worst = 0.0
    for lv in range(n_levels):
        f = lbm.lbm_get_populations_f64(g, lv)
        m = o.own[lv] == lv
        assert np.all(np.isfinite(f[:, m]))
        assert np.all(np.isnan(f[:, ~m]))
        ref = o.f[lv][:, m]
        worst = max(worst, float(np.max(np.abs(f[:, m] - ref) / np.abs(ref))))
    return worst


LMAP3 = np.array([2, 1, 0, 1], np.uint8).reshape(4, 1, 1)
LMAP2 = np.array([1, 0, 0, 1], np.uint8).reshape(4, 1, 1)


@pytest.mark.parametrize("schedule", ["disaggregated", "monolithic"])
def test_two_level_parity(lbm, schedule):
    g, dims, cell = make_mr(lbm, LMAP2, 2, 0.6, schedule)
    o = omr.MultiRes(LMAP2, 2, cell, 0.6)
    init_both(lbm, g, o, level_fields(dims, 2, 60))
    lbm.lbm_step(g, 50)               # 100 level-0 substeps
    o.run(50)
    assert compare(lbm, g, o, 2) <= F32_RTOL


@pytest.mark.parametrize("collision", ["bgk", "reg"])
def test_three_level_parity(lbm, collision):
    g, dims, cell = make_mr(lbm, LMAP3, 3, 0.58, collision=collision)
    o = omr.MultiRes(LMAP3, 3, cell, 0.58, collision)
    init_both(lbm, g, o, level_fields(dims, 3, 61))
    lbm.lbm_step(g, 25)               # 100 level-0 substeps
    o.run(25)
    assert compare(lbm, g, o, 3) <= F32_RTOL


def test_layout_bit_exact(lbm):
    lmap = np.zeros((4, 2, 2), np.uint8)
    lmap[:, 0, 0] = [2, 1, 0, 1]
    lmap[:, 1, 1] = [1, 1, 0, 1]
    lmap[:, 0, 1] = [2, 1, 1, 1]
    lmap[:, 1, 0] = [1, 1, 1, 1]
    g, dims, cell = make_mr(lbm, lmap, 3, 0.6)
    tab = olayout.multires_tables(lmap, 3, cell)
    info = lbm.lbm_get_info(g)
    for lv in range(3):
        t = tab[lv]
        assert info["n_group_b"][lv] == t["n_c"]
        assert info["n_blocks"][lv] == len(t["coords"])
        get = lambda what: lbm.lbm_get_layout(g, lv, what)
        assert get(lbm.LBM_LAYOUT_BLOCK_COORDS).tobytes() == t["coords"].tobytes()
        assert get(lbm.LBM_LAYOUT_NBR).tobytes() == t["nbr"].tobytes()
        assert get(lbm.LBM_LAYOUT_XNBR_COARSE).tobytes() == t["xnbr_coarse"].tobytes()
        assert get(lbm.LBM_LAYOUT_XNBR_FINE).tobytes() == t["xnbr_fine"].tobytes()


def test_fused_equals_unfused_bit_exact(lbm):
    fields = level_fields((32, 32, 128), 3, 62)
    out = []
    for sched in ("disaggregated", "monolithic"):
        g, dims, cell = make_mr(lbm, LMAP3, 3, 0.6, sched)
        for lv, (rho, u) in enumerate(fields):
            lbm.lbm_init_equilibrium(g, lv, rho, u)
        lbm.lbm_step(g, 6)
        out.append([lbm.lbm_get_populations_f64(g, lv) for lv in range(3)])
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)


def test_schedule_switches_and_streams_keep_results(lbm):
    """Switching between the fused and unfused schedules between calls, and
    stepping on a caller's stream with no synchronisation before the
    readback, give the populations of an all-fused run bit for bit: every
    level stream of a call is joined into the caller's stream, and a call
    orders after the work already on it."""
    import torch
    fields = level_fields((32, 32, 128), 3, 64)
    ref, _, _ = make_mr(lbm, LMAP3, 3, 0.6)
    for lv, (rho, u) in enumerate(fields):
        lbm.lbm_init_equilibrium(ref, lv, rho, u)
    lbm.lbm_step(ref, 6)
    want = [lbm.lbm_get_populations_f64(ref, lv) for lv in range(3)]
    g, _, _ = make_mr(lbm, LMAP3, 3, 0.6)
    for lv, (rho, u) in enumerate(fields):
        lbm.lbm_init_equilibrium(g, lv, rho, u)
    side = torch.cuda.Stream()
    lbm.lbm_step(g, 2, side)
    lbm.lbm_set_schedule(g, "monolithic")
    lbm.lbm_step(g, 1, side)
    lbm.lbm_set_schedule(g, "disaggregated")
    lbm.lbm_step(g, 2, side)
    lbm.lbm_step(g, 1)  # back on the grid's own stream
    for lv in range(3):
        assert np.array_equal(lbm.lbm_get_populations_f64(g, lv), want[lv], equal_nan=True)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_volume_weighted_conservation(lbm, storage):
    g, dims, cell = make_mr(lbm, LMAP3, 3, 0.6, storage=storage)
    for lv, (rho, u) in enumerate(level_fields(dims, 3, 63)):
        lbm.lbm_init_equilibrium(g, lv, rho, u)
    m0 = lbm.lbm_conservation(g)
    lbm.lbm_step(g, 10)
    m1 = lbm.lbm_conservation(g)
    tol = 1e-6 if storage == "f32" else 2e-5
    assert abs(m1[0] - m0[0]) / m0[0] <= tol
    assert np.all(np.abs(m1[1:] - m0[1:]) <= tol * m0[0])


def test_uniform_state_stays_uniform(lbm):
    g, dims, cell = make_mr(lbm, LMAP3, 3, 0.57)
    for lv in range(3):
        nx, ny, nz = (d >> lv for d in dims)
        u = np.zeros((3, nz, ny, nx))
        u[:] = np.array([0.02, -0.01, 0.03])[:, None, None, None]
        lbm.lbm_init_equilibrium(g, lv, np.full((nz, ny, nx), 1.01), u)
    f0 = [lbm.lbm_get_populations_f64(g, lv) for lv in range(3)]
    lbm.lbm_step(g, 3)
    for lv in range(3):
        f = lbm.lbm_get_populations_f64(g, lv)
        m = np.isfinite(f0[lv][0])
        # 3 coarse steps = 12 finest updates, each within a few FP32 ulps (3e-8 at 1/3)
        assert np.max(np.abs(f[:, m] - f0[lv][:, m])) < 1e-6


def test_full_size_three_level_turbulence_properties(lbm):
    """256^3 virtual finest box, level 0 = slab z in [96,160), level 1 = z in
    [64,96) u [160,192), level 2 elsewhere (the turbulence workload's layout)."""
    lmap = wl.multires_slab_map()
    g, dims, cell = make_mr(lbm, lmap, 3, 0.52)
    info = lbm.lbm_get_info(g)
    assert info["n_updated"] == [256 * 256 * 64, 128 * 128 * 32, 64 * 64 * 32]
    for lv in range(3):
        nx, ny, nz = (d >> lv for d in dims)
        rho, u = wl.random_fields((nz, ny, nx), seed=70 + lv, u_amp=0.02)
        lbm.lbm_init_equilibrium(g, lv, rho, u)
    m0 = lbm.lbm_conservation(g)
    lbm.lbm_step(g, 4)
    m1 = lbm.lbm_conservation(g)
    assert abs(m1[0] - m0[0]) / m0[0] <= 1e-6
    assert np.all(np.abs(m1[1:] - m0[1:]) <= 1e-6 * m0[0])
    lbm.lbm_sync(g)


# ------------------------------------------- lid-driven cavity (Sec. 6.3)

def make_cavity(lbm, n, n_levels, shells, tau, schedule="disaggregated", lid=True):
    lmap = wl.multires_cavity_map(n, n_levels, shells)
    g = lbm.lbm_grid_create_multires((n,) * 3, n_levels, lmap, lbm.physics(
        tau, "bgk", "f32", (0, 0, 0), schedule))
    flags, bc = wl.cavity(n)
    if not lid:
        flags = np.zeros_like(flags)
    lbm.lbm_set_boundary(g, 0, flags, bc_list(flags, bc) if lid else None)
    cell = 8 * 2 ** (n_levels - 1)
    o = omr.MultiRes(lmap, n_levels, cell, tau, periodic=(False,) * 3, flags0=flags,
                     bc0=oracle_bc(flags, bc) if lid else None)
    return g, o


def cavity_fields(n, n_levels, seed):
    rho, u = wl.random_fields((n,) * 3, seed=seed, u_amp=0.02)
    out = [(rho, u)]
    for _ in range(1, n_levels):
        rho, u = omr.subcell_mean(rho), omr.subcell_mean(u)
        out.append((rho, u))
    return out


@pytest.mark.parametrize("schedule", ["disaggregated", "monolithic"])
def test_cavity_two_level_parity(lbm, schedule):
    """Walls and the regularized lid on level 0, level 1 in the middle; 50
    coarsest steps (100 level-0 substeps)."""
    g, o = make_cavity(lbm, 48, 2, (1,), 0.6, schedule)
    init_both(lbm, g, o, cavity_fields(48, 2, 70))
    lbm.lbm_step(g, 50)
    o.run(50)
    assert compare(lbm, g, o, 2) <= F32_RTOL


def test_cavity_three_level_parity(lbm):
    """The smallest 3-level cavity the shell rule allows (160^3, level 2 in
    the central 32^3), one coarsest step (four level-0 substeps)."""
    g, o = make_cavity(lbm, 160, 3, (1, 1), 0.56)
    init_both(lbm, g, o, cavity_fields(160, 3, 71))
    lbm.lbm_step(g, 1)
    o.run(1)
    assert compare(lbm, g, o, 3) <= F32_RTOL


def test_cavity_fused_equals_unfused_and_closed_box_mass(lbm):
    out = []
    for schedule in ("disaggregated", "monolithic"):
        g, _ = make_cavity(lbm, 160, 3, (1, 1), 0.56, schedule)
        for lv, (r, u) in enumerate(cavity_fields(160, 3, 72)):
            lbm.lbm_init_equilibrium(g, lv, r, u)
        lbm.lbm_step(g, 3)
        out.append([lbm.lbm_get_populations_f64(g, lv) for lv in range(3)])
    for a, b in zip(*out):
        assert np.array_equal(np.nan_to_num(a, nan=-1.0), np.nan_to_num(b, nan=-1.0))
    g, _ = make_cavity(lbm, 160, 3, (1, 1), 0.56, lid=False)
    for lv, (r, u) in enumerate(cavity_fields(160, 3, 73)):
        lbm.lbm_init_equilibrium(g, lv, r, u)
    m0 = lbm.lbm_conservation(g)[0]
    lbm.lbm_step(g, 10)
    assert abs(lbm.lbm_conservation(g)[0] / m0 - 1) <= 1e-6


def test_cavity_rules_are_enforced(lbm):
    with pytest.raises(lbm.LbmError) as e:                # coarse cells on a wall
        lbm.lbm_grid_create_multires((32, 32, 32), 2, np.ones((2, 2, 2), np.uint8),
                                     lbm.physics(0.6, periodic=(0, 1, 1)))
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    lmap = wl.multires_cavity_map(48, 2, (1,))
    g = lbm.lbm_grid_create_multires((48,) * 3, 2, lmap, lbm.physics(0.6))
    flags = np.zeros((48,) * 3, np.uint8)
    flags[15, 20, 20] = wl.SOLID                           # in a G_c block of level 0
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_boundary(g, 0, flags)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("q", [19, 27])
def test_interface_voxel_lists_bit_exact(lbm, q):
    """The per-level interface voxel lists (slot and the bit set of the
    populations taken from another level) equal the oracle's, on maps with
    face, edge and corner contacts and on the cavity's nested shells."""
    lmap = np.zeros((4, 2, 2), np.uint8)
    lmap[:, 0, 0] = [2, 1, 0, 1]
    lmap[:, 1, 1] = [1, 1, 0, 1]
    lmap[:, 0, 1] = [2, 1, 1, 1]
    lmap[:, 1, 0] = [1, 1, 1, 1]
    cases = [(lmap, 3, (1, 1, 1)), (LMAP3, 3, (1, 1, 1)), (LMAP2, 2, (1, 1, 1)),
             (wl.multires_cavity_map(160, 3, (1, 1)), 3, (0, 0, 0))]
    for m, n_levels, per in cases:
        cell = 8 * 2 ** (n_levels - 1)
        mz, my, mx = m.shape
        g = lbm.lbm_grid_create_multires((mx * cell, my * cell, mz * cell), n_levels, m,
                                         lbm.physics(0.6, periodic=per, lattice=q))
        want = olayout.multires_interface(m, n_levels, cell, q=q)
        for lv in range(n_levels):
            slots = lbm.lbm_get_layout(g, lv, lbm.LBM_LAYOUT_IFACE_SLOTS)
            cross = lbm.lbm_get_layout(g, lv, lbm.LBM_LAYOUT_IFACE_CROSS)
            assert slots.tobytes() == want[lv][0].tobytes(), (m.shape, lv)
            assert cross.tobytes() == want[lv][1].tobytes(), (m.shape, lv)
        lbm.lbm_grid_destroy(g)


def test_staged_lean_kernel_equals_default(lbm):
    """Multi-resolution lean launches with each 8^3 block staged in shared
    memory by a bulk copy give the default kernel's populations bit for bit
    (3-level periodic map, and the 2-level cavity with walls and the lid on
    level 0)."""
    fields = level_fields((32, 32, 128), 3, 65)
    out = []
    for variant in (lbm.LBM_VARIANT_SCALAR, lbm.LBM_VARIANT_STAGED):
        g, _, _ = make_mr(lbm, LMAP3, 3, 0.6)
        lbm.lbm_set_variant(g, variant)
        for lv, (rho, u) in enumerate(fields):
            lbm.lbm_init_equilibrium(g, lv, rho, u)
        lbm.lbm_step(g, 4)
        out.append([lbm.lbm_get_populations_f64(g, lv) for lv in range(3)])
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)
    out = []
    for variant in (lbm.LBM_VARIANT_SCALAR, lbm.LBM_VARIANT_STAGED):
        g, o = make_cavity(lbm, 48, 2, (1,), 0.6)
        lbm.lbm_set_variant(g, variant)
        for lv, (r, u) in enumerate(cavity_fields(48, 2, 74)):
            lbm.lbm_init_equilibrium(g, lv, r, u)
        lbm.lbm_step(g, 4)
        out.append([lbm.lbm_get_populations_f64(g, lv) for lv in range(2)])
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)


def test_checkpoint_restore_into_new_grid_bit_exact(lbm):
    """Between coarsest steps a multi-resolution state is each level's
    current buffer: a snapshot of every level, restored into a freshly built
    grid, continues bit for bit like the original (the ring buffers of the
    previous step are not needed)."""
    import torch
    fields = level_fields((32, 32, 128), 3, 66)
    g, _, _ = make_mr(lbm, LMAP3, 3, 0.6)
    for lv, (rho, u) in enumerate(fields):
        lbm.lbm_init_equilibrium(g, lv, rho, u)
    lbm.lbm_step(g, 3)
    info = lbm.lbm_get_info(g)
    snaps = []
    for lv in range(3):
        snap = torch.empty(info["population_bytes"][lv], dtype=torch.uint8, device="cuda")
        lbm.lbm_get_populations(g, lv, snap)
        snaps.append(snap)
    lbm.lbm_step(g, 3)
    want = [lbm.lbm_get_populations_f64(g, lv) for lv in range(3)]
    h, _, _ = make_mr(lbm, LMAP3, 3, 0.6)
    for lv in range(3):
        lbm.lbm_set_populations(h, lv, snaps[lv])
    lbm.lbm_step(h, 3)
    for lv in range(3):
        assert np.array_equal(lbm.lbm_get_populations_f64(h, lv), want[lv], equal_nan=True)


LMAP4 = np.array([3, 2, 1, 0, 1, 2], np.uint8).reshape(6, 1, 1)


def test_four_level_parity_and_tables(lbm):
    """Four levels (refinement 2 at every jump, coarsest cell 64 finest
    voxels): interface voxel lists bit for bit, populations after one
    coarsest step (8 level-0 substeps) within 1e-5 of the oracle, and the
    unfused schedule equal to the fused one bit for bit."""
    g, dims, cell = make_mr(lbm, LMAP4, 4, 0.6)
    want = olayout.multires_interface(LMAP4, 4, cell)
    for lv in range(4):
        assert lbm.lbm_get_layout(g, lv, lbm.LBM_LAYOUT_IFACE_SLOTS).tobytes() == want[lv][0].tobytes()
        assert lbm.lbm_get_layout(g, lv, lbm.LBM_LAYOUT_IFACE_CROSS).tobytes() == want[lv][1].tobytes()
    o = omr.MultiRes(LMAP4, 4, cell, 0.6)
    fields = level_fields(dims, 4, 67)
    init_both(lbm, g, o, fields)
    lbm.lbm_step(g, 1)
    o.run(1)
    assert compare(lbm, g, o, 4) <= F32_RTOL
    u, _, _ = make_mr(lbm, LMAP4, 4, 0.6, "monolithic")
    for lv, (rho, v) in enumerate(fields):
        lbm.lbm_init_equilibrium(u, lv, rho, v)
    lbm.lbm_step(u, 1)
    for lv in range(4):
        assert np.array_equal(lbm.lbm_get_populations_f64(u, lv), lbm.lbm_get_populations_f64(g, lv),
                              equal_nan=True)
