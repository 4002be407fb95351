"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one oracle function to the mathematics of the lattice or to
a closed-form flow, so that a dropped term, a wrong sign, a wrong index or a
reversed shift anywhere in ``oracle/`` fails at least one of them.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from oracle import lattice as L
from oracle import lbm
from oracle import layout
from paper_2503_07898_gb300 import workloads as wl


# ------------------------------------------------------------------ lattice

def test_velocity_set_is_d3q19():
    """D3Q19 = every vector of {-1,0,1}^3 with |c|^2 <= 2 (19 of them)."""
    want = {c for c in itertools.product((-1, 0, 1), repeat=3) if sum(v * v for v in c) <= 2}
    got = {tuple(int(v) for v in c) for c in L.C}
    assert len(L.C) == 19 and got == want
    # opposite: c_opp(i) = -c_i and odd/even pairing of the chosen ordering
    for i in range(19):
        assert tuple(L.C[L.OPP[i]]) == tuple(-L.C[i])
        if i >= 1:
            assert L.OPP[i] == (i + 1 if i % 2 == 1 else i - 1)


def test_weights_isotropy_exact():
    """Moment isotropy of the weights in exact rational arithmetic."""
    w = L.W_FRAC
    c = [tuple(int(v) for v in ci) for ci in L.C]
    d = lambda a, b: 1 if a == b else 0
    assert sum(w) == 1
    for a in range(3):
        assert sum(w[i] * c[i][a] for i in range(19)) == 0
        for b in range(3):
            assert sum(w[i] * c[i][a] * c[i][b] for i in range(19)) == Fraction(d(a, b), 3)
            for g in range(3):
                assert sum(w[i] * c[i][a] * c[i][b] * c[i][g] for i in range(19)) == 0
                for e in range(3):
                    s = sum(w[i] * c[i][a] * c[i][b] * c[i][g] * c[i][e] for i in range(19))
                    want = Fraction(d(a, b) * d(g, e) + d(a, g) * d(b, e) + d(a, e) * d(b, g), 9)
                    assert s == want
    assert np.allclose(L.W, [float(x) for x in w], rtol=0, atol=0)


def test_equilibrium_moments():
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.1 * rng.random(50)
    u = 0.1 * (2 * rng.random((3, 50)) - 1)
    feq = L.equilibrium(rho, u)
    r, uu = L.moments(feq)
    assert np.allclose(r, rho, rtol=1e-15, atol=0)
    assert np.allclose(uu, u, rtol=0, atol=1e-15)
    pi = L.second_moment(feq)
    for a in range(3):
        for b in range(3):
            want = rho * ((1.0 / 3.0 if a == b else 0.0) + u[a] * u[b])
            assert np.allclose(pi[a, b], want, rtol=0, atol=2e-16)


def test_regularized_projection_reproduces_second_moment():
    """sum_i c_i c_i f^{neq,reg}_i = Pi for symmetric Pi; zero mass and momentum."""
    rng = np.random.default_rng(2)
    a = rng.standard_normal((3, 3, 7))
    pi = a + a.transpose(1, 0, 2)
    fneq = L.regularized_neq(pi)
    assert np.allclose(L.second_moment(fneq), pi, atol=1e-14)
    assert np.allclose(fneq.sum(axis=0), 0.0, atol=1e-14)
    assert np.allclose(L.C.T.astype(float) @ fneq, 0.0, atol=1e-14)


def test_reg_collision_equals_bgk_on_a_regularized_input():
    """Populations f^eq(rho, u) + f^{neq,reg}(Pi) have no non-equilibrium
    part outside the second-order Hermite space the regularized collision
    keeps, so REG and BGK give the same post-collision state, the closed form
    f^eq + (1 - 1/tau) f^{neq,reg}(Pi) (Latt and Chopard, Sec. 6.2)."""
    rng = np.random.default_rng(13)
    shape = (5, 6)
    rho = 1.0 + 0.02 * rng.standard_normal(shape)
    u = 0.03 * rng.standard_normal((3,) + shape)
    a = 1e-3 * rng.standard_normal((3, 3) + shape)
    pi = a + a.transpose(1, 0, 2, 3)
    g = L.equilibrium(rho, u) + L.regularized_neq(pi)
    for tau in (0.52, 0.6, 1.3):
        fb, _, _ = lbm.collide(g, tau, "bgk")
        fr, _, _ = lbm.collide(g, tau, "reg")
        want = L.equilibrium(rho, u) + (1.0 - 1.0 / tau) * L.regularized_neq(pi)
        assert np.allclose(fr, fb, rtol=0, atol=1e-15)
        assert np.allclose(fr, want, rtol=0, atol=1e-15)


def test_initial_state_fills_every_updated_voxel():
    """The initial state is f^eq(rho, u) on fluid voxels and on both kinds of
    regularized node, 0 on solid and not-in-domain voxels; its mass is the
    sum of rho over those updated voxels."""
    shape = (4, 5, 6)
    rho, u = wl.random_fields(shape, seed=15)
    flags = np.zeros(shape, np.uint8)
    flags[1, 2, 3] = wl.SOLID
    flags[:, :, 0] = wl.flag(wl.VELOCITY, wl.NX_M)
    flags[:, :, 5] = wl.flag(wl.PRESSURE, wl.NX_P)
    flags[0, 0, 0] = wl.OUTSIDE
    kept = np.ones(shape, bool)
    kept[1, 2, 3] = kept[0, 0, 0] = False
    f = lbm.init_equilibrium(rho, u, flags)
    assert np.array_equal(f[:, kept], L.equilibrium(rho, u)[:, kept])
    assert np.all(f[:, ~kept] == 0)
    assert abs(lbm.conservation(f)[0] - rho[kept].sum()) < 1e-12


# ------------------------------------------------------------ conservation

@pytest.mark.parametrize("collision", ["bgk", "reg"])
def test_periodic_mass_momentum_exact(collision):
    shape = (9, 10, 12)
    rho, u = wl.random_fields(shape, seed=11)
    flags = np.zeros(shape, dtype=np.uint8)
    f = lbm.init_equilibrium(rho, u)
    m0 = lbm.conservation(f)
    f = lbm.run(f, flags, 0.6, 100, collision=collision, periodic=(True, True, True))
    m1 = lbm.conservation(f)
    assert abs(m1[0] - m0[0]) / m0[0] <= 1e-13
    assert np.all(np.abs(m1[1:] - m0[1:]) <= 1e-13 * m0[0])


def test_uniform_flow_is_stationary():
    shape = (5, 6, 7)
    rho = np.full(shape, 1.02)
    u = np.zeros((3,) + shape)
    u[:] = np.array([0.03, -0.02, 0.01])[:, None, None, None]
    f0 = lbm.init_equilibrium(rho, u)
    f = lbm.run(f0, np.zeros(shape, np.uint8), 0.55, 10, periodic=(True, True, True))
    assert np.max(np.abs(f - f0)) < 1e-15


def test_centroid_moves_by_momentum():
    """One step moves the density centroid by exactly the momentum (sum_x x rho(t+1)
    - sum_x x rho(t) = J); a reversed streaming shift gives -J."""
    shape = (16, 16, 16)
    rho = np.ones(shape)
    u = np.zeros((3,) + shape)
    rng = np.random.default_rng(3)
    core = (slice(6, 10),) * 3
    rho[core] += 0.05 * rng.random((4, 4, 4))
    u[(slice(None),) + core] = 0.04 * rng.random((3, 4, 4, 4))
    f = lbm.init_equilibrium(rho, u)
    flags = np.zeros(shape, np.uint8)
    J = lbm.conservation(f)[1:]
    f1 = lbm.step(f, flags, 0.7, periodic=(True, True, True))
    r0, r1 = f.sum(0) - 1.0, f1.sum(0) - 1.0     # subtract the uniform background
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    for coord, a in ((x, 0), (y, 1), (z, 2)):
        shift = (coord * r1).sum() - (coord * r0).sum()
        assert abs(shift - J[a]) < 1e-11


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_step_commutes_with_a_shift_along_the_periodic_axis(axis):
    """With only `axis` periodic (bounce-back walls on the other two), the
    update commutes with a cyclic shift of the box along that axis; an axis
    treated as walled, or a wall taken for a periodic side, breaks it at the
    box ends."""
    shape = (6, 7, 8)
    rho, u = wl.random_fields(shape, seed=14 + axis)
    f = lbm.init_equilibrium(rho, u)
    flags = np.zeros(shape, np.uint8)
    periodic = tuple(a == axis for a in range(3))
    ax = 3 - axis                                 # populations are (q, z, y, x)
    a = lbm.step(np.roll(f, 1, axis=ax), flags, 0.6, periodic=periodic)
    b = np.roll(lbm.step(f, flags, 0.6, periodic=periodic), 1, axis=ax)
    assert np.allclose(a, b, rtol=0, atol=1e-15)
    # along a walled axis the same shift does not commute
    other = 3 - (axis + 1) % 3
    c = lbm.step(np.roll(f, 1, axis=other), flags, 0.6, periodic=periodic)
    d = np.roll(lbm.step(f, flags, 0.6, periodic=periodic), 1, axis=other)
    assert np.max(np.abs(c - d)) > 1e-6


# ---------------------------------------------------------- bounce-back

def test_closed_box_conserves_mass():
    shape = (7, 8, 9)
    rho, u = wl.random_fields(shape, seed=5)
    flags = np.zeros(shape, np.uint8)
    flags[3, 3:5, 4] = wl.SOLID
    f = lbm.init_equilibrium(rho, u, flags)
    m0 = lbm.conservation(f, flags)[0]
    f = lbm.run(f, flags, 0.58, 60)
    assert abs(lbm.conservation(f, flags)[0] - m0) / m0 < 1e-13


def test_not_in_domain_voxels_bounce_back_like_solids():
    """Voxels outside the domain (type 7) are walls (halfway bounce-back,
    Sec. 6.2): a fluid region enclosed by a shell of them on a periodic box
    conserves its mass exactly, and steps exactly as the same region
    enclosed by solid voxels."""
    shape = (8, 9, 10)
    rho, u = wl.random_fields(shape, seed=12)
    shell = np.ones(shape, bool)
    shell[1:-1, 1:-1, 1:-1] = False
    res = []
    for kind in (wl.OUTSIDE, wl.SOLID):
        flags = np.zeros(shape, np.uint8)
        flags[shell] = kind
        f = lbm.init_equilibrium(rho, u, flags)
        m0 = lbm.conservation(f, flags)[0]
        f = lbm.run(f, flags, 0.6, 40, periodic=(True, True, True))
        assert abs(lbm.conservation(f, flags)[0] - m0) / m0 < 1e-13
        res.append(f)
    assert np.array_equal(res[0], res[1])


def test_closed_box_mirror_symmetry():
    """A mirror-symmetric start in a closed box stays mirror-symmetric."""
    shape = (6, 7, 10)
    rho, u = wl.random_fields(shape, seed=6)
    rho = 0.5 * (rho + rho[:, :, ::-1])
    ux = 0.5 * (u[0] - u[0][:, :, ::-1])
    uy = 0.5 * (u[1] + u[1][:, :, ::-1])
    uz = 0.5 * (u[2] + u[2][:, :, ::-1])
    u = np.stack([ux, uy, uz])
    f = lbm.run(lbm.init_equilibrium(rho, u), np.zeros(shape, np.uint8), 0.6, 20)
    r, v = lbm.state_moments(f)
    assert np.allclose(r, r[:, :, ::-1], atol=1e-14)
    assert np.allclose(v[0], -v[0][:, :, ::-1], atol=1e-14)
    assert np.allclose(v[1], v[1][:, :, ::-1], atol=1e-14)


# ------------------------------------------------------------- closed forms

def test_taylor_green_decay():
    """Config-1 flow: 32^3 periodic 2D Taylor-Green, tau = 0.6, 100 steps.

    The amplitude decays as exp(-2 nu k^2 t) once the start-up transient of an
    equilibrium initial state has passed; the rate over steps 50..100 matches
    to 1e-3 and E/E0 after 100 steps to 2e-2 (the transient costs ~1.2 %).
    """
    n, tau = 32, 0.6
    rho, u = wl.taylor_green_2d(n)
    f = lbm.init_equilibrium(rho, u)
    flags = np.zeros((n, n, n), np.uint8)
    k = 2 * np.pi / n
    x = np.arange(n)
    mode = np.sin(k * x)[None, :] * np.cos(k * x)[:, None]

    def amp(f):
        _, v = lbm.state_moments(f)
        return (v[1, 0] * mode).sum() / (mode * mode).sum(), v

    def energy(f):
        r, v = lbm.state_moments(f)
        return 0.5 * (r * (v * v).sum(0)).sum()

    e0 = energy(f)
    f = lbm.run(f, flags, tau, 50, periodic=(True, True, True))
    a50, _ = amp(f)
    f = lbm.run(f, flags, tau, 50, periodic=(True, True, True))
    a100, v = amp(f)
    nu = (tau - 0.5) / 3
    rate = np.log(a100 / a50) / 50
    assert abs(rate / (-2 * nu * k * k) - 1) < 1e-3
    assert abs(energy(f) / e0 / lbm.tgv_energy_ratio(tau, k, 100) - 1) < 2e-2
    assert np.max(np.abs(v[2])) < 1e-15


def test_poiseuille_body_force_exact_at_magic_tau():
    """Halfway bounce-back is exact for Poiseuille flow at tau = 1/2 + sqrt(3/16)."""
    H = 16
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    g = 1e-6
    flags = np.zeros((1, H, 2), np.uint8)
    f = lbm.init_equilibrium(np.ones((1, H, 2)), np.zeros((3, 1, H, 2)))
    for _ in range(4000):
        f, rho, u = lbm.step(f, flags, tau, periodic=(True, False, True), force=(g, 0, 0),
                             return_macro=True)
    want = lbm.poiseuille_profile(g, (tau - 0.5) / 3, H)
    assert np.max(np.abs(u[0, 0, :, 0] / want - 1)) < 1e-8


def test_poiseuille_regularized_inlet_outlet():
    """Regularized velocity inlet (parabola) + regularized pressure outlet give
    the parabolic profile and the linear density drop 3 dp/dx = -24 nu u_max / H^2."""
    H, NX = 8, 24
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3
    umax = 1e-3
    y = np.arange(H)
    prof = umax * 4 * (y + 0.5) * (H - 0.5 - y) / H ** 2
    flags = np.zeros((1, H, NX), np.uint8)
    flags[:, :, 0] = wl.flag(wl.VELOCITY, wl.NX_M)
    flags[:, :, NX - 1] = wl.flag(wl.PRESSURE, wl.NX_P)
    bc = np.zeros((4, 1, H, NX))
    bc[3] = 1.0
    bc[0, 0, :, 0] = prof
    f = lbm.init_equilibrium(np.ones((1, H, NX)), np.zeros((3, 1, H, NX)))
    for _ in range(2500):
        f, rho, u = lbm.step(f, flags, tau, periodic=(False, False, True), bc=bc,
                             return_macro=True)
    mid = NX // 2
    assert np.max(np.abs(u[0, 0, :, mid] / prof - 1)) < 2e-3
    assert np.max(np.abs(u[1, 0, :, mid])) < 1e-8
    drho = (rho[0, H // 2, NX - 4] - rho[0, H // 2, 3]) / (NX - 7)
    assert abs(drho / (-24 * nu * umax / H ** 2) - 1) < 1e-2


# ---------------------------------------------------- regularized boundary

@pytest.mark.parametrize("normal", range(6))
@pytest.mark.parametrize("kind", [wl.VELOCITY, wl.PRESSURE])
def test_regularized_boundary_fixed_points(normal, kind):
    """Equilibrium and regularized non-equilibrium inputs are reproduced:
    g = f^eq + 9/2 w Q:Pi  ->  f* = f^eq + (1 - 1/tau) 9/2 w Q:Pi."""
    rng = np.random.default_rng(10 + normal)
    n = 5
    nvec = L.NORMALS[normal]
    rho = 1.0 + 0.05 * rng.random(n)
    u = 0.05 * (2 * rng.random((3, n)) - 1)
    if kind == wl.PRESSURE:
        un = u.T @ nvec
        u = np.outer(nvec, un)
    bc = np.vstack([u, rho[None]])
    tau = 0.57
    feq = L.equilibrium(rho, u)
    fs, r, uu = lbm.regularized_boundary(feq.copy(), normal, bc, kind, tau)
    assert np.allclose(fs, feq, atol=1e-15)
    assert np.allclose(r, rho, atol=1e-15)
    a = 1e-3 * rng.standard_normal((3, 3, n))
    pi = a + a.transpose(1, 0, 2)
    fneq = L.regularized_neq(pi)
    fs, r, _ = lbm.regularized_boundary(feq + fneq, normal, bc, kind, tau)
    assert np.allclose(r, rho, atol=1e-14)
    assert np.allclose(fs, feq + (1 - 1 / tau) * fneq, atol=1e-15)


def test_lid_nodes_carry_prescribed_velocity():
    """After one step every lid node (edges and corners included) stores
    populations whose velocity is exactly the prescribed lid velocity."""
    flags, bc = wl.cavity(4)
    rho, u = wl.random_fields((4, 4, 4), seed=12)
    f = lbm.init_equilibrium(rho, u)
    out = lbm.step(f, flags, 0.6, bc=bc)
    _, ulid = lbm.state_moments(out)
    assert np.allclose(ulid[:, 3], bc[:3, 3], atol=1e-15)


# ------------------------------------------------------------------ layout

def test_morton_code_values():
    assert layout.morton_code(1, 0, 0) == 1
    assert layout.morton_code(0, 1, 0) == 2
    assert layout.morton_code(0, 0, 1) == 4
    assert layout.morton_code(1, 1, 1) == 7
    assert layout.morton_code(2, 0, 0) == 8
    assert layout.morton_code(3, 5, 6) == 427
    cube = sorted(itertools.product(range(2), repeat=3), key=lambda c: layout.morton_code(*c))
    assert cube == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def test_block_tables_hand_example():
    flags = np.full((8, 16, 24), wl.OUTSIDE, np.uint8)
    flags[:, 0:16, 0:16] = wl.FLUID            # blocks (0,0,0),(1,0,0),(0,1,0),(1,1,0)
    flags[2, 3, 3] = wl.SOLID
    flags[5, 12, 12] = wl.flag(wl.VELOCITY, wl.NZ_P)   # block (1,1,0) is boundary
    flags[0, 0, 20] = wl.SOLID                  # block (2,0,0) holds only a solid voxel
    t = layout.block_tables(flags, 8)
    assert t["n_boundary"] == 1
    assert [tuple(c) for c in t["coords"]] == [(1, 1, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    k = lambda dx, dy, dz: (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
    nbr = t["nbr"]
    assert nbr[1, k(1, 0, 0)] == 2 and nbr[1, k(0, 1, 0)] == 3 and nbr[1, k(1, 1, 0)] == 0
    assert nbr[1, k(-1, 0, 0)] == -1 and nbr[2, k(1, 0, 0)] == -1
    assert nbr[0, k(0, 0, 0)] == 0


def test_block_tables_periodic_wrap_hand_example():
    """3 x 3 x 2 blocks, periodic along x and z, walls at the y sides:
    across a periodic side the neighbour is the block on the far side
    (with two blocks along z, -z and +z name the same block), across a
    walled side there is none, and the table is an involution."""
    flags = np.zeros((16, 24, 24), np.uint8)
    t = layout.block_tables(flags, 8, periodic=(True, False, True))
    ids = {tuple(int(v) for v in c): b for b, c in enumerate(t["coords"])}
    nbr = t["nbr"]
    k = lambda dx, dy, dz: (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
    b0 = ids[(0, 0, 0)]
    assert nbr[b0, k(-1, 0, 0)] == ids[(2, 0, 0)]
    assert nbr[b0, k(1, 0, 0)] == ids[(1, 0, 0)]
    assert nbr[b0, k(0, 0, -1)] == ids[(0, 0, 1)] == nbr[b0, k(0, 0, 1)]
    assert nbr[b0, k(-1, 0, -1)] == ids[(2, 0, 1)]
    assert nbr[b0, k(0, -1, 0)] == -1 and nbr[b0, k(-1, -1, 1)] == -1
    assert nbr[b0, k(1, 1, 1)] == ids[(1, 1, 1)]
    b1 = ids[(2, 2, 1)]
    assert nbr[b1, k(1, 0, 1)] == ids[(0, 2, 0)]
    assert nbr[b1, k(0, 1, 0)] == -1 and nbr[b1, k(0, -1, 0)] == ids[(2, 1, 1)]
    # the 6 blocks on each walled side miss the 9 neighbours across it
    assert len(ids) == 18 and int((nbr < 0).sum()) == 2 * 6 * 9
    for b in range(len(ids)):
        for kk in range(27):
            if nbr[b, kk] >= 0:
                assert nbr[nbr[b, kk], 26 - kk] == b


def test_block_tables_ragged_box_keeps_partial_blocks():
    """A 12 x 9 x 10 all-fluid box is cut into 2 x 2 x 2 blocks of 8^3 (the
    partial ones padded with not-in-domain voxels), every one active, in
    Morton order."""
    flags = np.zeros((10, 9, 12), np.uint8)
    t = layout.block_tables(flags, 8)
    assert [tuple(int(v) for v in c) for c in t["coords"]] == \
        [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    assert t["dims_blocks"] == (2, 2, 2) and t["n_boundary"] == 0


def test_block_tables_bitmask_grouping_hand_example():
    """Bitmask grouping of the example above: every block in Morton order,
    (1,1,0) marked by bit 3, its two regularized voxels indexed 0 and 1 in
    flag-scan order, every other slot -1."""
    flags = np.full((8, 16, 24), wl.OUTSIDE, np.uint8)
    flags[:, 0:16, 0:16] = wl.FLUID
    flags[5, 12, 12] = wl.flag(wl.VELOCITY, wl.NZ_P)
    flags[6, 9, 10] = wl.flag(wl.PRESSURE, wl.NX_M)
    t = layout.block_tables(flags, 8, grouping="bitmask")
    assert [tuple(c) for c in t["coords"]] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)]
    assert t["n_boundary"] == 1
    assert t["boundary_bits"].tolist() == [1 << 3]
    idx = t["bc_index"]
    # flag-scan order: (z=5, y=12, x=12) comes before (z=6, y=9, x=10)
    assert idx[3 * 512 + 4 + 8 * (4 + 8 * 5)] == 0
    assert idx[3 * 512 + 2 + 8 * (1 + 8 * 6)] == 1
    assert int((idx >= 0).sum()) == 2
    k = lambda dx, dy, dz: (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
    assert t["nbr"][0, k(1, 1, 0)] == 3 and t["nbr"][3, k(-1, 0, 0)] == 2


def test_block_tables_neighbour_symmetry_and_sphere_counts():
    """Config-3 geometry: 22 767 active 8^3 blocks (34.7 % of 65 536), 716 of
    them boundary (inlet + outlet columns); nbr is an involution."""
    flags, _ = wl.sphere_channel(dims=(512, 256, 256))
    t = flags & 7
    tb = t.reshape(32, 8, 32, 8, 64, 8)
    active = np.isin(tb, (0, 2, 3)).any(axis=(1, 3, 5))
    bound = np.isin(tb, (2, 3)).any(axis=(1, 3, 5))
    assert int(active.sum()) == 22767 and int(bound.sum()) == 716
    small = flags[96:160, 96:160, 0:64]
    tab = layout.block_tables(np.ascontiguousarray(small), 8)
    nbr = tab["nbr"]
    for b in range(len(nbr)):
        for kk in range(27):
            if nbr[b, kk] >= 0:
                assert nbr[nbr[b, kk], 26 - kk] == b


def test_multires_tables_hand_example():
    """Two levels side by side along x (periodic): level 0 owns x in [0,16),
    level 1 owns x in [16,32) of a 32 x 16 x 16 finest box."""
    t = layout.multires_tables(np.array([[[0, 1]]]), 2, 16)
    assert len(t[0]["coords"]) == 8 and t[0]["n_c"] == 8       # every level-0 block touches level 1
    assert [tuple(c) for c in t[0]["coords"]] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0),
                                                  (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    assert [tuple(c) for c in t[1]["coords"]] == [(1, 0, 0)] and t[1]["n_c"] == 1
    k = lambda dx, dy, dz: (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
    assert list(t[1]["xnbr_fine"][0, k(-1, 0, 0)]) == list(range(8))
    assert list(t[1]["xnbr_fine"][0, k(1, 0, 0)]) == list(range(8))
    assert t[1]["nbr"][0, k(0, 1, 0)] == 0 and t[1]["nbr"][0, k(1, 0, 0)] == -1
    # level-0 block (0,0,0): -x neighbour region is level 1 (periodic wrap), +x is level 0
    assert t[0]["xnbr_coarse"][0, k(-1, 0, 0)] == 0 and t[0]["nbr"][0, k(1, 0, 0)] == 1
    assert t[0]["xnbr_coarse"][1, k(1, 0, 0)] == 0


def test_multires_tables_coarse_neighbours_asymmetric_example():
    """Level 0 owns the map cell (x 0, y 0), level 1 the cells (1, 0),
    (0, 1) and (1, 1) of a 32 x 32 x 16 finest box (cells of 16 voxels).
    The level-1 blocks, all G_c, are numbered in Morton order: (1,0,0) = 0,
    (0,1,0) = 1, (1,1,0) = 2.  A level-0 block's coarse neighbour across
    +x, +y or the (+x, +y) edge is the level-1 block covering that region."""
    lmap = np.array([[[0, 1], [1, 1]]], np.uint8)
    t = layout.multires_tables(lmap, 2, 16)
    assert [tuple(int(v) for v in c) for c in t[1]["coords"]] == [(1, 0, 0), (0, 1, 0), (1, 1, 0)]
    ids = {tuple(int(v) for v in c): b for b, c in enumerate(t[0]["coords"])}
    xc = t[0]["xnbr_coarse"]
    k = lambda dx, dy, dz: (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
    assert xc[ids[(1, 0, 0)], k(1, 0, 0)] == 0
    assert xc[ids[(0, 1, 0)], k(0, 1, 0)] == 1
    assert xc[ids[(1, 1, 1)], k(1, 1, 0)] == 2
    assert xc[ids[(0, 0, 0)], k(-1, 0, 0)] == 0      # x wraps to the level-1 cell (1, 0)
    assert xc[ids[(0, 0, 0)], k(0, -1, 0)] == 1      # y wraps to the level-1 cell (0, 1)
    assert xc[ids[(1, 0, 0)], k(-1, 0, 0)] == -1     # (0,0,0) is level 0
    assert t[0]["nbr"][ids[(1, 0, 0)], k(-1, 0, 0)] == ids[(0, 0, 0)]


def test_multires_tables_interior_blocks_are_gi():
    """A thick fine slab: only the block layers touching the coarse level are G_c."""
    lmap = np.array([1, 0, 0, 1]).reshape(4, 1, 1)
    t = layout.multires_tables(lmap, 2, 32)
    # level 0 slab z in [32, 96): 8 block layers of 4x4 blocks; layers 4 and 11 touch level 1
    assert len(t[0]["coords"]) == 8 * 16 and t[0]["n_c"] == 2 * 16
    assert set(int(c[2]) for c in t[0]["coords"][:32]) == {4, 11}
