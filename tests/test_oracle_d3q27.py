"""Pins of the D3Q27 oracle: the same facts that pin D3Q19, for the lattice
the paper uses in its block-sparse register-pressure study (Sec. 6.2).

The oracle reads the lattice from the population count, so these tests run
the shared code of oracle/lbm.py on 27-population fields.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from oracle import lattice as L
from oracle import lbm
from paper_2503_07898_gb300 import workloads as wl

Q27 = L.D3Q27


def test_velocity_set_is_d3q27():
    """D3Q27 = all of {-1,0,1}^3; the first 19 are D3Q19 in the same order;
    opposites pair odd i with i + 1."""
    want = set(itertools.product((-1, 0, 1), repeat=3))
    got = {tuple(int(v) for v in c) for c in Q27.C}
    assert Q27.Q == 27 and got == want
    assert np.array_equal(Q27.C[:19], L.D3Q19.C)
    for i in range(27):
        assert tuple(Q27.C[Q27.OPP[i]]) == tuple(-Q27.C[i])
        if i >= 1:
            assert Q27.OPP[i] == (i + 1 if i % 2 == 1 else i - 1)


def test_weights_isotropy_exact():
    w = Q27.W_FRAC
    c = [tuple(int(v) for v in ci) for ci in Q27.C]
    d = lambda a, b: 1 if a == b else 0
    assert sum(w) == 1
    for a in range(3):
        assert sum(w[i] * c[i][a] for i in range(27)) == 0
        for b in range(3):
            assert sum(w[i] * c[i][a] * c[i][b] for i in range(27)) == Fraction(d(a, b), 3)
            for g in range(3):
                assert sum(w[i] * c[i][a] * c[i][b] * c[i][g] for i in range(27)) == 0
                for e in range(3):
                    s = sum(w[i] * c[i][a] * c[i][b] * c[i][g] * c[i][e] for i in range(27))
                    want = Fraction(d(a, b) * d(g, e) + d(a, g) * d(b, e) + d(a, e) * d(b, g), 9)
                    assert s == want
    # the weights of {c.n = 0} plus twice those of {c.n > 0} sum to 1 for
    # every axis normal (the shifted Zou-He density relies on it)
    for nvec in L.NORMALS:
        cn = Q27.C @ nvec
        assert sum(w[i] for i in range(27) if cn[i] == 0) + 2 * sum(
            w[i] for i in range(27) if cn[i] > 0) == 1


def test_equilibrium_and_projection_moments():
    rng = np.random.default_rng(31)
    rho = 1.0 + 0.1 * rng.random(40)
    u = 0.1 * (2 * rng.random((3, 40)) - 1)
    feq = Q27.equilibrium(rho, u)
    r, uu = L.moments(feq)
    assert np.allclose(r, rho, rtol=1e-15, atol=0)
    assert np.allclose(uu, u, rtol=0, atol=1e-15)
    pi = L.second_moment(feq)
    for a in range(3):
        for b in range(3):
            want = rho * ((1.0 / 3.0 if a == b else 0.0) + u[a] * u[b])
            assert np.allclose(pi[a, b], want, rtol=0, atol=2e-16)
    a = rng.standard_normal((3, 3, 7))
    p = a + a.transpose(1, 0, 2)
    fneq = Q27.regularized_neq(p)
    assert fneq.shape[0] == 27
    assert np.allclose(L.second_moment(fneq), p, atol=1e-14)
    assert np.allclose(fneq.sum(axis=0), 0.0, atol=1e-14)
    assert np.allclose(Q27.C.T.astype(float) @ fneq, 0.0, atol=1e-14)


@pytest.mark.parametrize("collision", ["bgk", "reg"])
def test_periodic_mass_momentum_exact(collision):
    shape = (7, 8, 9)
    rho, u = wl.random_fields(shape, seed=32)
    flags = np.zeros(shape, dtype=np.uint8)
    f = lbm.init_equilibrium(rho, u, q=27)
    m0 = lbm.conservation(f)
    f = lbm.run(f, flags, 0.6, 40, collision=collision, periodic=(True, True, True))
    assert f.shape[0] == 27
    m1 = lbm.conservation(f)
    assert abs(m1[0] - m0[0]) / m0[0] <= 1e-13
    assert np.all(np.abs(m1[1:] - m0[1:]) <= 1e-13 * m0[0])


def test_centroid_moves_by_momentum():
    shape = (12, 12, 12)
    rho = np.ones(shape)
    u = np.zeros((3,) + shape)
    rng = np.random.default_rng(33)
    core = (slice(4, 8),) * 3
    rho[core] += 0.05 * rng.random((4, 4, 4))
    u[(slice(None),) + core] = 0.04 * rng.random((3, 4, 4, 4))
    f = lbm.init_equilibrium(rho, u, q=27)
    J = lbm.conservation(f)[1:]
    f1 = lbm.step(f, np.zeros(shape, np.uint8), 0.7, periodic=(True, True, True))
    r0, r1 = f.sum(0) - 1.0, f1.sum(0) - 1.0
    z, y, x = np.meshgrid(np.arange(12), np.arange(12), np.arange(12), indexing="ij")
    for coord, a in ((x, 0), (y, 1), (z, 2)):
        assert abs((coord * r1).sum() - (coord * r0).sum() - J[a]) < 1e-11


def test_closed_box_with_obstacle_conserves_mass():
    shape = (6, 7, 8)
    rho, u = wl.random_fields(shape, seed=34)
    flags = np.zeros(shape, np.uint8)
    flags[2:4, 3, 3:5] = wl.SOLID
    f = lbm.init_equilibrium(rho, u, flags, q=27)
    m0 = lbm.conservation(f, flags)[0]
    f = lbm.run(f, flags, 0.58, 40)
    assert abs(lbm.conservation(f, flags)[0] - m0) / m0 < 1e-13


def test_taylor_green_decay_rate():
    """Viscosity (tau - 1/2)/3 on D3Q27: late-time decay rate of the 2D
    Taylor-Green mode to 1e-3."""
    n, tau = 24, 0.6
    rho, u = wl.taylor_green_2d(n)
    f = lbm.init_equilibrium(rho, u, q=27)
    flags = np.zeros((n, n, n), np.uint8)
    k = 2 * np.pi / n
    x = np.arange(n)
    mode = np.sin(k * x)[None, :] * np.cos(k * x)[:, None]

    def amp(f):
        _, v = lbm.state_moments(f)
        return (v[1, 0] * mode).sum() / (mode * mode).sum()

    f = lbm.run(f, flags, tau, 40, periodic=(True, True, True))
    a40 = amp(f)
    f = lbm.run(f, flags, tau, 40, periodic=(True, True, True))
    a80 = amp(f)
    rate = np.log(a80 / a40) / 40
    assert abs(rate / (-2 * (tau - 0.5) / 3 * k * k) - 1) < 1e-3


@pytest.mark.parametrize("normal", range(6))
@pytest.mark.parametrize("kind", [wl.VELOCITY, wl.PRESSURE])
def test_regularized_boundary_fixed_points(normal, kind):
    rng = np.random.default_rng(40 + normal)
    n = 4
    nvec = L.NORMALS[normal]
    rho = 1.0 + 0.05 * rng.random(n)
    u = 0.05 * (2 * rng.random((3, n)) - 1)
    if kind == wl.PRESSURE:
        u = np.outer(nvec, u.T @ nvec)
    bc = np.vstack([u, rho[None]])
    tau = 0.57
    feq = Q27.equilibrium(rho, u)
    fs, r, _ = lbm.regularized_boundary(feq.copy(), normal, bc, kind, tau)
    assert np.allclose(fs, feq, atol=1e-15) and np.allclose(r, rho, atol=1e-15)
    a = 1e-3 * rng.standard_normal((3, 3, n))
    fneq = Q27.regularized_neq(a + a.transpose(1, 0, 2))
    fs, r, _ = lbm.regularized_boundary(feq + fneq, normal, bc, kind, tau)
    assert np.allclose(r, rho, atol=1e-14)
    assert np.allclose(fs, feq + (1 - 1 / tau) * fneq, atol=1e-15)


def test_poiseuille_regularized_inlet_outlet():
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
    f = lbm.init_equilibrium(np.ones((1, H, NX)), np.zeros((3, 1, H, NX)), q=27)
    for _ in range(2500):
        f, rho, u = lbm.step(f, flags, tau, periodic=(False, False, True), bc=bc,
                             return_macro=True)
    mid = NX // 2
    assert np.max(np.abs(u[0, 0, :, mid] / prof - 1)) < 2e-3
    drho = (rho[0, H // 2, NX - 4] - rho[0, H // 2, 3]) / (NX - 7)
    assert abs(drho / (-24 * nu * umax / H ** 2) - 1) < 1e-2


# ------------------------------------------------------ multi-resolution

def _mr(lmap, n_levels, cell, tau, **kw):
    from oracle import multires as mr
    return mr.MultiRes(np.asarray(lmap), n_levels, cell, tau, q=27, **kw)


def _init_random(g, seed):
    for lv in range(g.L):
        nx, ny, nz = g.dims(lv)
        rho, u = wl.random_fields((nz, ny, nx), seed=seed + lv)
        g.init_equilibrium(lv, rho, u)


@pytest.mark.parametrize("collision", ["bgk", "reg"])
def test_multires_volume_weighted_conservation_exact(collision):
    """Corner directions cross the level jumps too: mass and momentum,
    weighted by voxel volume, are still conserved exactly."""
    g = _mr(np.array([2, 1, 0, 1]).reshape(4, 1, 1), 3, 8, 0.6, collision=collision)
    _init_random(g, 160)
    m0 = g.conservation()
    g.run(4)
    m1 = g.conservation()
    assert g.f[0].shape[0] == 27
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-12
    assert np.all(np.abs(m1[1:] - m0[1:]) < 1e-12 * m0[0])


def test_multires_uniform_state_is_stationary():
    g = _mr(np.array([2, 1, 0, 1]).reshape(4, 1, 1), 3, 8, 0.57)
    for lv in range(3):
        nx, ny, nz = g.dims(lv)
        u = np.zeros((3, nz, ny, nx))
        u[:] = np.array([0.02, -0.01, 0.03])[:, None, None, None]
        g.init_equilibrium(lv, np.full((nz, ny, nx), 1.01), u)
    f0 = [a.copy() for a in g.f]
    g.run(3)
    for a, b in zip(f0, g.f):
        assert np.max(np.abs(a - b)) < 1e-15


def test_multires_single_level_equals_plain_oracle():
    g = _mr(np.zeros((1, 1, 1), int), 1, 12, 0.6)
    rho, u = wl.random_fields((12, 12, 12), seed=161)
    g.init_equilibrium(0, rho, u)
    g.run(4)
    ref = lbm.run(lbm.init_equilibrium(rho, u, q=27), np.zeros((12, 12, 12), np.uint8), 0.6, 4,
                  periodic=(True, True, True))
    assert np.max(np.abs(g.f[0] - ref)) < 1e-15


def test_multires_cavity_near_walls_equals_single_resolution():
    from oracle import multires as mr
    n, T = 48, 3
    lmap = wl.multires_cavity_map(n, 2, (1,))
    flags, bc = wl.cavity(n)
    rho, u = wl.random_fields((n,) * 3, seed=162, u_amp=0.02)
    g = _mr(lmap, 2, 16, 0.6, periodic=(False,) * 3, flags0=flags, bc0=bc)
    g.init_equilibrium(0, rho, u)
    g.init_equilibrium(1, mr.subcell_mean(rho), mr.subcell_mean(u))
    g.run(T)
    ref = lbm.run(lbm.init_equilibrium(rho, u, flags, q=27), flags, 0.6, 2 * T, bc=bc)
    c = np.arange(n)
    d1 = np.maximum(np.maximum(16 - c, c - 31), 0)
    dist = np.maximum(np.maximum(d1[:, None, None], d1[None, :, None]), d1[None, None, :])
    far = dist > 2 * T + 4
    assert np.max(np.abs(g.f[0][:, far] - ref[:, far])) < 1e-15


def test_multires_tables_count_corner_neighbours():
    """A level-0 block that meets level 1 only across a block corner is G_c
    for D3Q27 and G_i for D3Q19."""
    from oracle import layout
    lmap = np.zeros((2, 2, 2), np.uint8)
    lmap[1, 1, 1] = 1                       # one coarse cell at the far corner
    t19 = layout.multires_tables(lmap, 2, 16, q=19)
    t27 = layout.multires_tables(lmap, 2, 16, q=27)
    assert t27[0]["n_c"] > t19[0]["n_c"]
