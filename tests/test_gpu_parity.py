"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Every case builds its inputs with ``workloads`` (seeded), runs the library
and the oracle on the same inputs, and compares populations of every updated
voxel element by element (max relative error <= 1e-5 after 100 FP32 steps).
Sizes span several CTA tiles with ragged tails; full-size configurations are
checked on sampled voxels that the oracle computes one by one.
"""
import numpy as np
import pytest

from cases import (F32_RTOL, make_grid, max_rel_err, oracle_window, run_oracle, updated_mask,
                   velocity_l2)
from oracle import layout as olayout
from oracle import lbm as olbm
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def gpu_run(lbm, g, rho, u, steps):
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, steps)
    return lbm.lbm_get_populations_f64(g, 0)


# ------------------------------------------------------------------ dense

def test_taylor_green_config1(lbm):
    """32^3 periodic Taylor-Green, tau 0.6, BGK, FP32, 100 steps."""
    n, tau = 32, 0.6
    rho, u = wl.taylor_green_2d(n)
    flags = np.zeros((n, n, n), np.uint8)
    g = make_grid(lbm, "dense", flags, None, tau, periodic=(1, 1, 1))
    f = gpu_run(lbm, g, rho, u, 100)
    ref = run_oracle(flags, None, rho, u, tau, 100, periodic=(1, 1, 1))
    assert max_rel_err(f, ref, flags) <= F32_RTOL
    # kinetic energy against the closed form (start-up transient included)
    r, v = lbm.lbm_get_moments(g, 0)
    e = 0.5 * (r * (v * v).sum(0)).sum()
    e0 = 0.5 * (rho * (u * u).sum(0)).sum()
    assert abs(e / e0 / olbm.tgv_energy_ratio(tau, 2 * np.pi / n, 100) - 1) < 2e-2


@pytest.mark.parametrize("collision", ["bgk", "reg"])
def test_dense_periodic_random_ragged(lbm, collision):
    dims_zyx = (13, 21, 45)
    rho, u = wl.random_fields(dims_zyx, seed=21)
    flags = np.zeros(dims_zyx, np.uint8)
    g = make_grid(lbm, "dense", flags, None, 0.6, collision, periodic=(1, 1, 1))
    f = gpu_run(lbm, g, rho, u, 100)
    ref = run_oracle(flags, None, rho, u, 0.6, 100, collision, periodic=(1, 1, 1))
    assert max_rel_err(f, ref, flags) <= F32_RTOL


@pytest.mark.parametrize("schedule", ["disaggregated", "monolithic"])
@pytest.mark.parametrize("tau", [0.6, 0.515])
def test_cavity_ragged(lbm, schedule, tau):
    """Lid-driven cavity (config-2 physics) on a ragged 37 x 19 x 23 box."""
    dims_zyx = (23, 19, 37)
    flags, bc = wl.cavity(0, dims=(37, 19, 23))
    rho, u = wl.random_fields(dims_zyx, seed=22, u_amp=0.02)
    g = make_grid(lbm, "dense", flags, bc, tau, schedule=schedule)
    f = gpu_run(lbm, g, rho, u, 100)
    ref = run_oracle(flags, bc, rho, u, tau, 100)
    assert max_rel_err(f, ref, flags) <= F32_RTOL


def test_cavity_schedules_agree(lbm):
    flags, bc = wl.cavity(0, dims=(40, 24, 16))
    rho, u = wl.random_fields(flags.shape, seed=23)
    out = []
    for sched in ("disaggregated", "monolithic"):
        g = make_grid(lbm, "dense", flags, bc, 0.55, schedule=sched)
        out.append(gpu_run(lbm, g, rho, u, 50))
    m = updated_mask(flags)
    assert np.max(np.abs(out[0][:, m] - out[1][:, m])) <= 1e-6


@pytest.mark.parametrize("schedule", ["disaggregated", "monolithic"])
def test_dense_channel_obstacles(lbm, schedule):
    """Regularized inlet / outlet (not a contiguous tail: per-voxel wall mask
    path), solid obstacles, bounce-back side walls."""
    dims_zyx = (14, 18, 41)
    flags = wl.random_obstacles(dims_zyx, seed=24, solid_fraction=0.08)
    flags[:, :, 0] = wl.flag(wl.VELOCITY, wl.NX_M)
    flags[:, :, -1] = wl.flag(wl.PRESSURE, wl.NX_P)
    bc = np.zeros((4,) + dims_zyx)
    bc[0, :, :, 0] = 0.03
    bc[3] = 1.0
    bc[3, :, :, -1] = 0.995
    rho, u = wl.random_fields(dims_zyx, seed=25, u_amp=0.02)
    g = make_grid(lbm, "dense", flags, bc, 0.58, schedule=schedule)
    f = gpu_run(lbm, g, rho, u, 100)
    ref = run_oracle(flags, bc, rho, u, 0.58, 100)
    assert max_rel_err(f, ref, flags) <= F32_RTOL


# ----------------------------------------------------------------- sparse

def small_sphere_channel():
    return wl.sphere_channel(dims=(76, 44, 44), radius_channel=19, sphere_center_x=22,
                             sphere_radius=8, u_in=0.04)


@pytest.mark.parametrize("block_edge", [8, 4])
@pytest.mark.parametrize("schedule", ["disaggregated", "monolithic", "bitmask"])
def test_sparse_sphere_channel(lbm, block_edge, schedule):
    flags, bc = small_sphere_channel()
    rho, u = wl.random_fields(flags.shape, seed=26, u_amp=0.02)
    g = make_grid(lbm, "sparse", flags, bc, 0.56, schedule=schedule, block_edge=block_edge)
    f = gpu_run(lbm, g, rho, u, 100)
    ref = run_oracle(flags, bc, rho, u, 0.56, 100)
    assert max_rel_err(f, ref, flags) <= F32_RTOL


@pytest.mark.parametrize("block_edge", [8, 4])
def test_sparse_layout_bit_exact(lbm, block_edge):
    flags, bc = small_sphere_channel()
    g = make_grid(lbm, "sparse", flags, bc, 0.56, block_edge=block_edge)
    tab = olayout.block_tables(flags, block_edge)
    coords = lbm.lbm_get_layout(g, 0, lbm.LBM_LAYOUT_BLOCK_COORDS).reshape(-1, 3)
    nbr = lbm.lbm_get_layout(g, 0, lbm.LBM_LAYOUT_NBR).reshape(-1, 27)
    assert coords.tobytes() == tab["coords"].tobytes()
    assert nbr.tobytes() == tab["nbr"].tobytes()
    info = lbm.lbm_get_info(g)
    assert info["n_group_b"][0] == tab["n_boundary"]
    assert info["n_updated"][0] == int(updated_mask(flags).sum())
    assert lbm.lbm_get_layout(g, 0, lbm.LBM_LAYOUT_FLAGS).tobytes() == flags.tobytes()


@pytest.mark.parametrize("block_edge", [8, 4])
def test_sparse_bitmask_layout_bit_exact(lbm, block_edge):
    """Bitmask grouping (Sec. 4, Table 2): Morton order over all blocks,
    boundary bits and the per-slot index of the compact boundary values equal
    the oracle's tables byte for byte."""
    flags, bc = small_sphere_channel()
    g = make_grid(lbm, "sparse", flags, bc, 0.56, schedule="bitmask", block_edge=block_edge)
    tab = olayout.block_tables(flags, block_edge, grouping="bitmask")
    coords = lbm.lbm_get_layout(g, 0, lbm.LBM_LAYOUT_BLOCK_COORDS).reshape(-1, 3)
    nbr = lbm.lbm_get_layout(g, 0, lbm.LBM_LAYOUT_NBR).reshape(-1, 27)
    assert coords.tobytes() == tab["coords"].tobytes()
    assert nbr.tobytes() == tab["nbr"].tobytes()
    bits = lbm.lbm_get_layout(g, 0, lbm.LBM_LAYOUT_BOUNDARY_BITS)
    assert bits.tobytes() == tab["boundary_bits"].tobytes()
    idx = lbm.lbm_get_layout(g, 0, lbm.LBM_LAYOUT_BC_INDEX)
    assert idx.tobytes() == tab["bc_index"].tobytes()
    assert lbm.lbm_get_info(g)["n_group_b"][0] == tab["n_boundary"] > 0


def test_sparse_bitmask_equals_memory_grouping(lbm):
    """Both groupings run the same per-voxel arithmetic: identical populations
    after 60 steps (FP32 and FP16 storage)."""
    flags, bc = small_sphere_channel()
    rho, u = wl.random_fields(flags.shape, seed=27, u_amp=0.02)
    for storage in ("f32", "f16"):
        out = []
        for schedule in ("disaggregated", "bitmask"):
            g = make_grid(lbm, "sparse", flags, bc, 0.56, storage=storage, schedule=schedule)
            out.append(gpu_run(lbm, g, rho, u, 60))
        m = updated_mask(flags)
        assert np.array_equal(out[0][:, m], out[1][:, m]), storage


def test_grouping_is_fixed_at_creation(lbm):
    flags, bc = small_sphere_channel()
    gb = make_grid(lbm, "sparse", flags, bc, 0.56, schedule="bitmask")
    lbm.lbm_set_schedule(gb, "monolithic")
    lbm.lbm_set_schedule(gb, "bitmask")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_schedule(gb, "disaggregated")
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    gm = make_grid(lbm, "sparse", flags, bc, 0.56)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_schedule(gm, "bitmask")
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_grid_create_dense((16, 16, 16), lbm.physics(0.6, schedule="bitmask"))
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_grid_create_multires((32, 32, 32), 2, np.zeros((1, 1, 1), np.uint8),
                                     lbm.physics(0.6, periodic=(1, 1, 1), schedule="bitmask"))
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


def test_step_without_boundary_values_is_rejected(lbm):
    """Regularized voxels with no boundary values: lbm_step refuses to run."""
    flags, _ = small_sphere_channel()
    nz, ny, nx = flags.shape
    for schedule in ("disaggregated", "bitmask"):
        g = lbm.lbm_grid_create_sparse((nx, ny, nz), 8, flags, lbm.physics(0.56, schedule=schedule))
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(g, 1)
        assert e.value.status == lbm.LBM_ERR_INVALID


def test_sparse_periodic_equals_dense(lbm):
    """A sparse grid with every block active reproduces the dense grid."""
    dims_zyx = (16, 24, 32)
    flags = np.zeros(dims_zyx, np.uint8)
    rho, u = wl.random_fields(dims_zyx, seed=27)
    gd = make_grid(lbm, "dense", flags, None, 0.6, periodic=(1, 1, 1))
    gs = make_grid(lbm, "sparse", flags, None, 0.6, periodic=(1, 1, 1))
    fd = gpu_run(lbm, gd, rho, u, 30)
    fs = gpu_run(lbm, gs, rho, u, 30)
    assert np.max(np.abs(fd - fs)) <= 1e-6


# ------------------------------------------------------- moments, reductions

def test_moments_and_conservation(lbm):
    dims_zyx = (12, 20, 36)
    rho, u = wl.random_fields(dims_zyx, seed=28)
    flags = np.zeros(dims_zyx, np.uint8)
    g = make_grid(lbm, "dense", flags, None, 0.6, periodic=(1, 1, 1))
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    m0 = lbm.lbm_conservation(g)
    ref0 = olbm.conservation(olbm.init_equilibrium(rho, u))
    assert abs(m0[0] / ref0[0] - 1) < 1e-7
    assert np.all(np.abs(m0[1:] - ref0[1:]) < 1e-6 * ref0[0])
    lbm.lbm_step(g, 100)
    m1 = lbm.lbm_conservation(g)
    assert abs(m1[0] - m0[0]) / m0[0] <= 1e-6
    assert np.all(np.abs(m1[1:] - m0[1:]) <= 1e-6 * m0[0])
    # bit-reproducible reduction
    assert np.array_equal(m1, lbm.lbm_conservation(g))
    r, v = lbm.lbm_get_moments(g, 0)
    ref = run_oracle(flags, None, rho, u, 0.6, 100, periodic=(1, 1, 1))
    rr, vr = olbm.state_moments(ref)
    assert np.max(np.abs(r / rr - 1)) < 1e-6
    # the field has decayed to |u| ~ 1e-3: bound the absolute error (populations
    # agree to 1e-5 relative, so |du| <~ 18 * 1e-5 * max f_i / rho)
    assert np.max(np.abs(v - vr)) < 1e-6
    assert velocity_l2(v, vr, flags) < 1e-3


def test_checkpoint_roundtrip_bit_exact(lbm):
    import torch
    flags, bc = wl.cavity(0, dims=(24, 20, 16))
    rho, u = wl.random_fields(flags.shape, seed=29)
    g = make_grid(lbm, "dense", flags, bc, 0.6)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, 10)
    nbytes = lbm.lbm_get_info(g)["population_bytes"][0]
    snap = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lbm.lbm_get_populations(g, 0, snap)
    lbm.lbm_step(g, 10)
    a = lbm.lbm_get_populations_f64(g, 0)
    lbm.lbm_set_populations(g, 0, snap)
    lbm.lbm_step(g, 10)
    b = lbm.lbm_get_populations_f64(g, 0)
    m = updated_mask(flags)
    assert np.array_equal(a[:, m], b[:, m])


def test_invalid_arguments(lbm):
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_grid_create_dense((8, 8, 8), lbm.physics(0.5))
    assert e.value.status == lbm.LBM_ERR_INVALID
    flags = np.zeros((8, 8, 8), np.uint8)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_grid_create_sparse((8, 8, 8), 5, flags, lbm.physics(0.6))
    assert e.value.status == lbm.LBM_ERR_INVALID
    g = lbm.lbm_grid_create_sparse((8, 8, 8), 8, flags, lbm.physics(0.6))
    bad = flags.copy()
    bad[0, 0, 0] = wl.SOLID
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_boundary(g, 0, bad)
    assert e.value.status == lbm.LBM_ERR_INVALID
    gd = lbm.lbm_grid_create_dense((8, 8, 8), lbm.physics(0.6))
    lid = flags.copy()
    lid[-1] = wl.flag(wl.VELOCITY, wl.NZ_P)
    with pytest.raises(lbm.LbmError) as e:   # regularized voxels but no values
        lbm.lbm_set_boundary(gd, 0, lid)
    assert e.value.status == lbm.LBM_ERR_INVALID


# ------------------------------------------------ full-size sampled checks

def _sample_windows(lbm, g, flags, bc, rho, u, tau, steps, points):
    import torch
    nz, ny, nx = flags.shape
    dev = torch.empty((19, nz, ny, nx), dtype=torch.float64, device="cuda")
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, steps)
    lbm.lbm_get_populations_f64(g, 0, dev)
    worst = 0.0
    for p in points:
        got = dev[:, p[0], p[1], p[2]].cpu().numpy()
        ref = oracle_window(flags, bc, rho, u, p, steps, tau)
        worst = max(worst, float(np.max(np.abs(got - ref) / np.abs(ref))))
    del dev
    return worst


def test_full_size_cavity_config2_sampled(lbm):
    """256^3 cavity, tau 0.515, lid 0.05, seeded random start; 4 steps;
    voxels at lid corners and edges, walls and interior vs the oracle."""
    n = 256
    flags, bc = wl.cavity(n)
    rho, u = wl.random_fields((n, n, n), seed=30, u_amp=0.02)
    g = make_grid(lbm, "dense", flags, bc, 0.515)
    pts = [(255, 0, 0), (255, 255, 255), (255, 128, 0), (255, 17, 200), (0, 0, 0),
           (0, 255, 128), (128, 128, 128), (254, 3, 251), (100, 0, 77), (31, 200, 255)]
    assert _sample_windows(lbm, g, flags, bc, rho, u, 0.515, 4, pts) <= F32_RTOL


def test_full_size_sphere_config3_sampled(lbm):
    """512 x 256 x 256 sparse sphere channel, 8^3 blocks; 4 steps; voxels at the
    inlet, outlet, sphere surface, channel wall and bulk vs the oracle."""
    flags, bc = wl.sphere_channel()
    rho, u = wl.random_fields(flags.shape, seed=31, u_amp=0.02)
    g = make_grid(lbm, "sparse", flags, bc, 0.52)
    info = lbm.lbm_get_info(g)
    assert info["n_blocks"][0] == 22767 and info["n_group_b"][0] == 716
    pts = [(128, 128, 0), (128, 128, 511), (128, 48, 0), (128, 128, 95), (128, 160, 128),
           (128, 128, 161), (200, 128, 300), (128, 48, 300), (80, 80, 511), (128, 208, 7)]
    for p in pts:
        assert updated_mask(flags)[p], p
    assert _sample_windows(lbm, g, flags, bc, rho, u, 0.52, 4, pts) <= F32_RTOL


# -------------------------------------------- staged (bulk-copy) lean kernel

@pytest.mark.parametrize("storage,lattice", [("f32", 19), ("f16", 19), ("bf16", 19), ("f32", 27)])
def test_staged_variant_equals_default_kernel(lbm, storage, lattice):
    """The lean kernel that stages each 8^3 block in shared memory by one bulk
    copy reads the same values as the default kernel: identical populations
    after 40 steps of the sphere channel (walls, missing neighbour blocks,
    regularized inlet / outlet in the other group), and FP32 D3Q19 within
    1e-5 of the oracle."""
    flags, bc = small_sphere_channel()
    rho, u = wl.random_fields(flags.shape, seed=28, u_amp=0.02)
    out = []
    for variant in (lbm.LBM_VARIANT_SCALAR, lbm.LBM_VARIANT_STAGED):
        g = make_grid(lbm, "sparse", flags, bc, 0.56, storage=storage, lattice=lattice)
        lbm.lbm_set_variant(g, variant)
        out.append(gpu_run(lbm, g, rho, u, 40))
        lbm.lbm_sync(g)
    m = updated_mask(flags)
    assert np.array_equal(out[0][:, m], out[1][:, m])
    if storage == "f32" and lattice == 19:
        ref = run_oracle(flags, bc, rho, u, 0.56, 40)
        assert max_rel_err(out[1], ref, flags) <= F32_RTOL


def test_staged_variant_rejected_where_it_does_not_apply(lbm):
    flags = np.zeros((8, 8, 8), np.uint8)
    g = make_grid(lbm, "dense", flags, None, 0.6)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_variant(g, lbm.LBM_VARIANT_STAGED)
    g = make_grid(lbm, "sparse", flags, None, 0.6, block_edge=4)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_variant(g, lbm.LBM_VARIANT_STAGED)


def test_pinned_host_arrays_match_pageable(lbm):
    """Page-locked host arrays are read and written by the kernels in place;
    the results equal those of pageable arrays (staged through device
    scratch) bit for bit."""
    import torch
    flags, bc = wl.cavity(0, dims=(24, 20, 16))
    rho, u = wl.random_fields(flags.shape, seed=30, u_amp=0.02)
    out = []
    for pinned in (False, True):
        g = make_grid(lbm, "dense", flags, bc, 0.6)
        if pinned:
            r = torch.from_numpy(np.ascontiguousarray(rho)).pin_memory()
            v = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
            lbm.lbm_init_equilibrium(g, 0, r, v)
        else:
            lbm.lbm_init_equilibrium(g, 0, rho, u)
        lbm.lbm_step(g, 5)
        if pinned:
            ro = torch.empty(flags.size, dtype=torch.float64).pin_memory()
            uo = torch.empty(3 * flags.size, dtype=torch.float64).pin_memory()
            lbm.lbm_get_moments(g, 0, ro, uo)
            out.append((ro.numpy().reshape(flags.shape), uo.numpy().reshape((3,) + flags.shape)))
        else:
            out.append(lbm.lbm_get_moments(g, 0))
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)
