"""Pins of the multi-resolution oracle (oracle/multires.py).

The paper gives no explosion / coalescence formulas, so these pins tie the
reading to what must hold for any correct scheme of this family: exact
volume-weighted conservation, invariance of a uniform state, reduction to
the single-resolution oracle away from level jumps, and the viscous decay
rate of a Taylor-Green vortex crossing a level jump.
"""
import numpy as np
import pytest

from oracle import closure as ocl
from oracle import lattice as L
from oracle import lbm as olbm
from oracle import multires as mr
from paper_2503_07898_gb300 import workloads as wl


def three_level(tau0=0.6):
    # z-slabs of 8 finest voxels: level 2, 1, 0, 1 (periodic in z)
    return mr.MultiRes(np.array([2, 1, 0, 1]).reshape(4, 1, 1), 3, 8, tau0)


def init_random(g, seed):
    for lv in range(g.L):
        nx, ny, nz = g.dims(lv)
        rho, u = wl.random_fields((nz, ny, nx), seed=seed + lv)
        g.init_equilibrium(lv, rho, u)


@pytest.mark.parametrize("collision", ["bgk", "reg"])
def test_volume_weighted_conservation_exact(collision):
    g = three_level()
    g.collision = collision
    init_random(g, 50)
    m0 = g.conservation()
    g.run(6)
    m1 = g.conservation()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-12
    assert np.all(np.abs(m1[1:] - m0[1:]) < 1e-12 * m0[0])


def test_uniform_state_is_stationary():
    g = three_level(0.57)
    for lv in range(3):
        nx, ny, nz = g.dims(lv)
        rho = np.full((nz, ny, nx), 1.01)
        u = np.zeros((3, nz, ny, nx))
        u[:] = np.array([0.02, -0.01, 0.03])[:, None, None, None]
        g.init_equilibrium(lv, rho, u)
    f0 = [a.copy() for a in g.f]
    g.run(3)
    for a, b in zip(f0, g.f):
        assert np.max(np.abs(a - b)) < 1e-15


def test_single_level_equals_plain_oracle():
    g = mr.MultiRes(np.zeros((1, 1, 1), int), 1, 12, 0.6)
    rho, u = wl.random_fields((12, 12, 12), seed=51)
    g.init_equilibrium(0, rho, u)
    g.run(5)
    ref = olbm.run(olbm.init_equilibrium(rho, u), np.zeros((12, 12, 12), np.uint8), 0.6, 5,
                   periodic=(True, True, True))
    assert np.max(np.abs(g.f[0] - ref)) < 1e-15
    # every region on level 1: a plain coarse run with tau_1
    g = mr.MultiRes(np.ones((2, 1, 1), int), 2, 8, 0.6)
    rho, u = wl.random_fields((8, 4, 4), seed=52)
    g.init_equilibrium(1, rho, u)
    g.run(4)
    ref = olbm.run(olbm.init_equilibrium(rho, u), np.zeros((8, 4, 4), np.uint8),
                   mr.tau_of_level(0.6, 1), 4, periodic=(True, True, True))
    assert np.max(np.abs(g.f[1] - ref)) < 1e-15


def block_mean(a):
    return mr.subcell_mean(a)


def test_far_field_equals_single_resolution():
    """Coarse voxels beyond the light cone of the level jump evolve exactly as
    in a pure coarse run; fine voxels likewise as in a pure fine run."""
    # coarse far field: fine slab z in [16, 24) of a 48-voxel column
    lmap = np.array([1, 1, 0, 1, 1, 1]).reshape(6, 1, 1)
    g = mr.MultiRes(lmap, 2, 8, 0.6)
    rho_f, u_f = wl.random_fields((48, 8, 8), seed=53)
    rho_c, u_c = block_mean(rho_f), block_mean(u_f)
    g.init_equilibrium(0, rho_f, u_f)
    g.init_equilibrium(1, rho_c, u_c)
    n = 2
    g.run(n)
    ref = olbm.run(olbm.init_equilibrium(rho_c, u_c), np.zeros(rho_c.shape, np.uint8),
                   mr.tau_of_level(0.6, 1), n, periodic=(True, True, True))
    # coarse z index range of the fine slab: [8, 12); far = distance >= n + 2
    far = [z for z in range(24) if min(abs(z - 8), abs(z - 11), 24 - abs(z - 8)) >= n + 2
           and not 8 <= z < 12]
    assert far
    assert np.max(np.abs(g.f[1][:, far] - ref[:, far])) < 1e-14
    # fine far field: fine slab z in [8, 32)
    lmap = np.array([1, 0, 0, 0, 1, 1]).reshape(6, 1, 1)
    g = mr.MultiRes(lmap, 2, 8, 0.6)
    g.init_equilibrium(0, rho_f, u_f)
    g.init_equilibrium(1, rho_c, u_c)
    g.run(1)
    ref = olbm.run(olbm.init_equilibrium(rho_f, u_f), np.zeros(rho_f.shape, np.uint8), 0.6, 2,
                   periodic=(True, True, True))
    far = list(range(8 + 5, 32 - 5))
    assert np.max(np.abs(g.f[0][:, far] - ref[:, far])) < 1e-14


def test_taylor_green_across_level_jump():
    """A z-uniform Taylor-Green vortex on two levels (z slabs) decays at the
    viscous rate -2 nu k^2 on both levels (physical time, finest units)."""
    n = 32
    lmap = np.broadcast_to(np.array([0, 0, 1, 1]).reshape(4, 1, 1), (4, 2, 2))
    g = mr.MultiRes(lmap, 2, 16, 0.6)
    rho_f, u_f = wl.taylor_green_2d(n, u0=0.01, dims=(n, n, 64))
    g.init_equilibrium(0, rho_f, u_f)
    g.init_equilibrium(1, block_mean(rho_f), block_mean(u_f))
    k = 2 * np.pi / n
    nu = (0.6 - 0.5) / 3

    def layer_amps(lv):
        nx, ny, nz = g.dims(lv)
        x = (np.arange(nx) + 0.5) * 2 ** lv - 0.5     # voxel centres in finest units
        mode = np.sin(k * x)[None, :] * np.cos(k * x)[:, None]
        _, v = olbm.state_moments(g.f[lv])
        return np.array([(v[1][z] * mode).sum() / (mode * mode).sum() for z in range(nz)])

    g.run(20)
    a20 = [layer_amps(0)[:32], layer_amps(1)[16:]]
    g.run(20)
    a40 = [layer_amps(0)[:32], layer_amps(1)[16:]]
    want = -2 * nu * k * k
    ratio = [np.log(b / a) / 40.0 / want for a, b in zip(a20, a40)]   # 20 coarse = 40 finest units
    # layers away from the level jump (>= 6 fine / 3 coarse voxels) decay at the viscous rate
    assert np.all(np.abs(ratio[0][6:26] - 1) < 1e-2), ratio[0]
    assert np.all(np.abs(ratio[1][3:13] - 1) < 1e-2), ratio[1]
    # next to the jump the plain volumetric transfer (no non-equilibrium
    # rescaling) damps faster, within a bounded band
    assert np.all(np.abs(ratio[0] - 1) < 0.25) and np.all(np.abs(ratio[1] - 1) < 0.25)
    assert np.all(np.isfinite(g.conservation()))


# ---------------------------------------------------------------- closure

def _net(b3=0.0):
    return np.concatenate([np.zeros(ocl.N_PARAMS - 1), [b3]])


def _plain(rho, u, tau, n):
    return olbm.run(olbm.init_equilibrium(rho, u), np.zeros(rho.shape, np.uint8), tau, n,
                    periodic=(True, True, True))


def test_closure_zero_network_changes_nothing():
    ref = three_level(0.58)
    init_random(ref, 53)
    ref.run(3)
    g = mr.MultiRes(np.array([2, 1, 0, 1]).reshape(4, 1, 1), 3, 8, 0.58, theta=_net())
    init_random(g, 53)
    g.run(3)
    for a, b in zip(ref.f, g.f):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("b3,level", [(0.03, 2), (-0.004, 1), (0.03, 0), (-1.0, 2)])
def test_closure_constant_output_shifts_tau_of_coarse_levels(b3, level):
    """A network with constant output b3 on a grid owned by one level: levels
    >= 1 run the plain oracle at max(tau_l + b3, 1/2 + 1e-3), level 0 at tau_0."""
    tau0 = 0.56
    g = mr.MultiRes(np.full((2, 1, 1), level), 3, 8, tau0, theta=_net(b3))
    nx, ny, nz = g.dims(level)
    rho, u = wl.random_fields((nz, ny, nx), seed=54 + level)
    g.init_equilibrium(level, rho, u)
    g.run(2)
    tau_l = mr.tau_of_level(tau0, level)
    tau = tau_l if level == 0 else max(tau_l + b3, 0.5 + 1e-3)
    ref = _plain(rho, u, tau, 2 ** (2 - level) * 2)
    assert np.max(np.abs(g.f[level] - ref)) < 1e-15


def test_closure_sees_tau_of_its_level():
    """Network d_tau = relu(relu(feature 15)) = tau_l: level 1 then relaxes
    with 2 tau_1."""
    th = ocl.unpack(_net())
    th["W1"][0, 15] = 1.0
    th["W2"][0, 0] = 1.0
    th["W3"][0] = 1.0
    g = mr.MultiRes(np.full((2, 1, 1), 1), 2, 8, 0.6, theta=ocl.pack(th))
    nx, ny, nz = g.dims(1)
    rho, u = wl.random_fields((nz, ny, nx), seed=56)
    g.init_equilibrium(1, rho, u)
    g.run(3)
    ref = _plain(rho, u, 2 * mr.tau_of_level(0.6, 1), 3)
    assert np.max(np.abs(g.f[1] - ref)) < 1e-15


def test_closure_keeps_volume_weighted_conservation():
    rng = np.random.default_rng(57)
    th = rng.standard_normal(ocl.N_PARAMS) * 0.05
    g = mr.MultiRes(np.array([2, 1, 0, 1]).reshape(4, 1, 1), 3, 8, 0.6, theta=th)
    init_random(g, 58)
    m0 = g.conservation()
    g.run(3)
    m1 = g.conservation()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-12
    assert np.all(np.abs(m1[1:] - m0[1:]) < 1e-12 * m0[0])


# ------------------------------------------------- walls on the finest level

def test_cavity_single_level_equals_plain_oracle():
    """Walls and a regularized lid on a one-level grid: the plain cavity."""
    n = 16
    flags, bc = wl.cavity(n)
    g = mr.MultiRes(np.zeros((1, 1, 1), int), 1, n, 0.6, periodic=(False,) * 3,
                    flags0=flags, bc0=bc)
    rho, u = wl.random_fields((n, n, n), seed=60)
    g.init_equilibrium(0, rho, u)
    g.run(5)
    ref = olbm.run(olbm.init_equilibrium(rho, u, flags), flags, 0.6, 5, bc=bc)
    assert np.max(np.abs(g.f[0] - ref)) < 1e-15


def test_coarse_cells_on_walls_are_rejected():
    with pytest.raises(ValueError):
        mr.MultiRes(np.ones((2, 2, 2), int), 2, 16, 0.6, periodic=(False, True, True))
    with pytest.raises(ValueError):
        flags = np.zeros((32, 32, 32), np.uint8)
        flags[20, 20, 20] = wl.SOLID                 # inside the level-1 region
        mr.MultiRes(np.array([0, 1]).reshape(2, 1, 1), 2, 16, 0.6, flags0=flags)


def test_closed_box_conserves_volume_weighted_mass():
    lmap = wl.multires_cavity_map(48, 2, (1,))     # level 1 in the central 16^3
    g = mr.MultiRes(lmap, 2, 16, 0.6, periodic=(False,) * 3)
    init_random(g, 61)
    m0 = g.conservation()[0]
    g.run(3)
    assert abs(g.conservation()[0] / m0 - 1) < 1e-12


def test_closed_box_with_an_obstacle_conserves_volume_weighted_mass():
    """Solid voxels on level 0 are walls: they bounce back and hold no
    populations, so the volume-weighted mass of the two-level closed box
    stays exact."""
    lmap = wl.multires_cavity_map(48, 2, (1,))
    flags0 = np.zeros((48, 48, 48), np.uint8)
    flags0[3:9, 20:26, 5:11] = wl.SOLID            # inside level 0's shell
    g = mr.MultiRes(lmap, 2, 16, 0.6, periodic=(False,) * 3, flags0=flags0)
    init_random(g, 63)
    assert np.all(g.f[0][:, flags0 == wl.SOLID] == 0)
    m0 = g.conservation()[0]
    g.run(3)
    assert np.all(g.f[0][:, flags0 == wl.SOLID] == 0)
    assert abs(g.conservation()[0] / m0 - 1) < 1e-12


def test_cavity_near_walls_equals_single_resolution():
    """Finest-level voxels beyond the light cone of the level jump (lid,
    walls and the edges between them) evolve exactly as in a plain fine
    cavity run of the same fine steps."""
    n, T = 48, 3
    lmap = wl.multires_cavity_map(n, 2, (1,))
    flags, bc = wl.cavity(n)
    rho, u = wl.random_fields((n,) * 3, seed=62, u_amp=0.02)
    g = mr.MultiRes(lmap, 2, 16, 0.6, periodic=(False,) * 3, flags0=flags, bc0=bc)
    g.init_equilibrium(0, rho, u)
    g.init_equilibrium(1, mr.subcell_mean(rho), mr.subcell_mean(u))
    g.run(T)
    ref = olbm.run(olbm.init_equilibrium(rho, u, flags), flags, 0.6, 2 * T, bc=bc)
    c = np.arange(n)
    d1 = np.maximum(np.maximum(16 - c, c - 31), 0)          # per-axis distance to [16, 31]
    dist = np.maximum(np.maximum(d1[:, None, None], d1[None, :, None]), d1[None, None, :])
    far = dist > 2 * T + 4
    assert far.sum() > 0.4 * n ** 3
    assert np.max(np.abs(g.f[0][:, far] - ref[:, far])) < 1e-15
    near = (dist > 0) & ~far
    assert np.max(np.abs(g.f[0][:, near] - ref[:, near])) > 1e-8   # the jump does reach them


# ------------------------------------ interface voxels (Sec. 5, P_d = 0)

def _exchange_dependence(lmap, n_levels, cell, lv, q):
    """Which populations of level lv the oracle's exchange reads from another
    level's buffers, found by running it: every other level holds NaN (the
    finer level also after each of its substeps), level lv holds ones,
    collision is the identity, and one step of level lv is taken; a
    population comes out NaN iff its pre-collision value read another level."""
    o = mr.MultiRes(lmap, n_levels, cell, 0.6, q=q)
    for k in range(n_levels):
        o.f[k][:] = 1.0 if k == lv else np.nan
    real_advance = o._advance

    def advance(level, k, f0_self):
        if level < lv:
            o.f[level][:] = np.nan
        else:
            real_advance(level, k, f0_self)

    o._advance = advance
    real = olbm.collide
    olbm.collide = lambda g, tau, collision="bgk", force=None: (g, None, None)
    try:
        o._advance(lv, 1, o.f[lv].copy())
    finally:
        olbm.collide = real
    mine = o.own[lv] == lv
    dep = np.zeros(mine.shape, np.uint32)
    for i in range(1, o.lat.Q):
        dep |= np.where(np.isnan(o.f[lv][i]) & mine, np.uint32(1 << i), np.uint32(0))
    return dep


@pytest.mark.parametrize("q", [19, 27])
def test_interface_voxels_match_the_exchange(q):
    """layout.multires_interface (a direct formula) against the exchange the
    multi-resolution oracle performs, on a map with face, edge and corner
    contacts between the three levels."""
    from oracle import layout as olayout
    lmap = np.zeros((4, 2, 2), np.uint8)
    lmap[:, 0, 0] = [2, 1, 0, 1]
    lmap[:, 1, 1] = [1, 1, 0, 1]
    lmap[:, 0, 1] = [2, 1, 1, 1]
    lmap[:, 1, 0] = [1, 1, 1, 1]
    cell = 32
    res = olayout.multires_interface(lmap, 3, cell, q=q)
    tabs = olayout.multires_tables(lmap, 3, cell, q=q)
    for lv in range(3):
        dep = _exchange_dependence(lmap, 3, cell, lv, q)
        slots, cross = res[lv]
        coords = tabs[lv]["coords"]
        b, v = slots // 512, slots % 512
        x = coords[b, 0] * 8 + v % 8
        y = coords[b, 1] * 8 + (v // 8) % 8
        z = coords[b, 2] * 8 + v // 64
        want = np.zeros_like(dep)
        want[z, y, x] = cross
        assert np.array_equal(want, dep), lv
        assert np.all(np.diff(slots) > 0)
        # every interface voxel lies in a G_c block, and a G_c block holds one
        assert np.array_equal(np.unique(b), np.arange(tabs[lv]["n_c"]))
