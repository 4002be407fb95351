"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only (flag fields, boundary values,
initial density and velocity fields).  It contains none of the
lattice-Boltzmann arithmetic: the equilibrium, streaming, boundaries and
collision live in the CUDA library (and, for testing, in the independent
oracle).  Both sides receive the same arrays from here.

Flag byte: bits 0-2 type (0 fluid, 1 solid, 2 regularized velocity,
3 regularized pressure, 7 not in domain); bits 3-5 outward normal index
(0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z).  Arrays are (nz, ny, nx), x fastest.
"""
import numpy as np

FLUID, SOLID, VELOCITY, PRESSURE, OUTSIDE = 0, 1, 2, 3, 7
NX_P, NX_M, NY_P, NY_M, NZ_P, NZ_M = 0, 1, 2, 3, 4, 5


def flag(kind, normal=0):
    return np.uint8((kind & 7) | ((normal & 7) << 3))


def cavity(n, u_lid=0.05, dims=None):
    """Lid-driven cavity (Sec. 6.1): closed box, top plane z = nz-1 is a
    regularized velocity node with outward normal +z moving at u_lid along x;
    the other five sides are halfway bounce-back walls (box edges).

    Returns (flags, bc) with bc of shape (4, nz, ny, nx) = (ux, uy, uz, rho).
    """
    nx, ny, nz = dims if dims is not None else (n, n, n)
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags[nz - 1] = flag(VELOCITY, NZ_P)
    bc = np.zeros((4, nz, ny, nx), dtype=np.float64)
    bc[0, nz - 1] = u_lid
    bc[3] = 1.0
    return flags, bc


def sphere_channel(dims=(512, 256, 256), radius_channel=81, sphere_center_x=128,
                   sphere_radius=32, u_in=0.04, rho_out=1.0):
    """Flow past a sphere in a circular channel (Sec. 6.2 wind-tunnel setup).

    Fluid iff (y-cy)^2 + (z-cz)^2 < Rc^2 and the voxel is outside the sphere;
    voxels outside the channel are 'not in domain', the sphere is solid.
    x = 0 is a regularized velocity inlet (normal -x, u = (u_in, 0, 0)),
    x = nx-1 a regularized pressure outlet (normal +x, rho = rho_out).
    """
    nx, ny, nz = dims
    cy, cz = ny // 2, nz // 2
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    in_channel = ((y - cy) ** 2 + (z - cz) ** 2) < radius_channel ** 2
    in_sphere = ((x - sphere_center_x) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) < sphere_radius ** 2
    in_channel = np.broadcast_to(in_channel, (nz, ny, nx))
    flags = np.full((nz, ny, nx), OUTSIDE, dtype=np.uint8)
    flags[in_channel] = FLUID
    flags[in_channel & in_sphere] = SOLID
    inlet = in_channel[:, :, 0]
    outlet = in_channel[:, :, nx - 1] & ~in_sphere[:, :, nx - 1]
    flags[:, :, 0][inlet & ~in_sphere[:, :, 0]] = flag(VELOCITY, NX_M)
    flags[:, :, nx - 1][outlet] = flag(PRESSURE, NX_P)
    bc = np.zeros((4, nz, ny, nx), dtype=np.float64)
    bc[0, :, :, 0] = u_in
    bc[3] = rho_out
    return flags, bc


def taylor_green_2d(n, u0=0.02, dims=None):
    """2D Taylor-Green vortex in a periodic box (x, y), uniform along z.

    u = -u0 cos(kx) sin(ky), v = u0 sin(kx) cos(ky), w = 0, k = 2 pi / n,
    rho = 1 - 3/4 u0^2 (cos 2kx + cos 2ky) (pressure of the exact solution,
    rho' = 3 p').  Voxel centres at integer coordinates.
    """
    nx, ny, nz = dims if dims is not None else (n, n, n)
    kx = 2.0 * np.pi / nx
    ky = 2.0 * np.pi / ny
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    shape = (nz, ny, nx)
    u = np.zeros((3,) + shape, dtype=np.float64)
    u[0] = np.broadcast_to(-u0 * np.cos(kx * x) * np.sin(ky * y), shape)
    u[1] = np.broadcast_to(u0 * np.sin(kx * x) * np.cos(ky * y), shape)
    rho = np.broadcast_to(1.0 - 0.75 * u0 * u0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y)),
                          shape).copy()
    return rho, u


def random_fields(shape_zyx, seed, rho_amp=0.01, u_amp=0.03):
    """Seeded random density / velocity fields (uniform noise around rest)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * (2.0 * rng.random(shape_zyx) - 1.0)
    u = u_amp * (2.0 * rng.random((3,) + tuple(shape_zyx)) - 1.0)
    return rho, u


def random_obstacles(shape_zyx, seed, solid_fraction=0.1, kind="spheres"):
    """Random solid spheres (or boxes) until ~solid_fraction of voxels are solid."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    flags = np.zeros(shape_zyx, dtype=np.uint8)
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    target = solid_fraction * flags.size
    tries = 0
    while (flags == SOLID).sum() < target and tries < 10000:
        tries += 1
        r = rng.integers(2, max(3, min(nx, ny, nz) // 6) + 1)
        c = [rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)]
        if kind == "spheres":
            m = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 < r * r
        else:
            m = (abs(x - c[0]) < r) & (abs(y - c[1]) < r) & (abs(z - c[2]) < r)
        flags[np.broadcast_to(m, shape_zyx)] = SOLID
    return flags


def multires_slab_map(n=256, n_levels=3):
    """Level map of the three-level decaying-turbulence workload: a 256^3
    virtual finest box, level 0 in the central slab z in [96, 160), level 1 in
    z in [64, 96) u [160, 192), level 2 elsewhere.  One map cell is the
    coarsest block (8 * 2^(n_levels-1) finest voxels); shape (mz, my, mx)."""
    cell = 8 * 2 ** (n_levels - 1)
    m = n // cell
    zlev = np.full(m, 2, np.uint8)
    z = (np.arange(m) * cell)
    zlev[(z >= 64) & (z < 96)] = 1
    zlev[(z >= 160) & (z < 192)] = 1
    zlev[(z >= 96) & (z < 160)] = 0
    return np.ascontiguousarray(np.broadcast_to(zlev[:, None, None], (m, m, m)))


def multires_cavity_map(n=384, n_levels=3, shells=(2, 2)):
    """Level map of a multi-resolution lid-driven cavity (the benchmark of
    Sec. 6.3, Table 5): level 0 along every box face, shells[0] map cells
    thick, then level 1 for shells[1] cells, and so on inwards, the coarsest
    level in the middle.  One map cell is the coarsest block (8 * 2^(L-1)
    finest voxels); shape (mz, my, mx).  The walls and the lid then lie on
    the finest level, as the library requires of non-periodic grids."""
    cell = 8 * 2 ** (n_levels - 1)
    m = n // cell
    i = np.arange(m)
    d = np.minimum(i, m - 1 - i)
    dist = np.minimum(np.minimum(d[:, None, None], d[None, :, None]), d[None, None, :])
    lv = np.full((m, m, m), n_levels - 1, np.uint8)
    edge = 0
    for level, t in enumerate(shells[:n_levels - 1]):
        lv[(dist >= edge) & (dist < edge + t)] = level
        edge += t
    return lv


def turbulence(n, seed=7898, u_rms=0.03, kmax=None, dims=None):
    """Decaying-turbulence start: random-phase Fourier modes on integer wave
    vectors 1 <= |k| <= kmax with shell amplitude sqrt(E(k) / shell count),
    E(k) ~ k^(-5/3), projected divergence-free, real part of the inverse FFT,
    scaled to a component RMS of u_rms; rho = 1.  Returns (rho, u)."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    kmax = kmax if kmax is not None else min(nx, ny, nz) // 8
    rng = np.random.default_rng(seed)
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    shell = np.rint(kk).astype(int)
    counts = np.bincount(shell.ravel())
    amp = np.zeros_like(kk)
    ok = (shell >= 1) & (kk <= kmax)
    amp[ok] = np.sqrt(shell[ok].astype(float) ** (-5.0 / 3.0) / counts[shell[ok]])
    uh = amp[None] * (rng.standard_normal((3,) + kk.shape) + 1j * rng.standard_normal((3,) + kk.shape))
    kvec = np.broadcast_arrays(kx, ky, kz)
    with np.errstate(invalid="ignore", divide="ignore"):
        kdotu = sum(kvec[a] * uh[a] for a in range(3)) / np.where(kk > 0, kk * kk, 1.0)
    for a in range(3):
        uh[a] = uh[a] - kvec[a] * kdotu
    u = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    u *= u_rms / np.sqrt(np.mean(u * u))
    return np.ones((nz, ny, nx)), u


def batch_cases(n_cases=128, seed=7898, lmin=32, lmax=160, max_solid=0.20, tau=(0.52, 0.8),
                u0=0.02, max_edge=None):
    """Serving-style batch: independent periodic cases, every edge drawn
    uniformly in [lmin, lmax] and rounded to a multiple of 8, even cases dense
    and odd cases 8^3 block-sparse, random solid spheres (or boxes) up to a
    drawn solid fraction in [0, max_solid], tau drawn in `tau`, a 2D
    Taylor-Green start of amplitude u0 (batch_case_fields).  Returns a list
    of dicts; with max_edge, only the cases whose largest edge is at most
    max_edge (the same cases, drawn from the same sequence)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cases):
        dims = tuple(int(8 * max(1, round(int(rng.integers(lmin, lmax + 1)) / 8))) for _ in range(3))
        frac = float(rng.uniform(0.0, max_solid))
        tau_c = float(rng.uniform(*tau))
        if max_edge is not None and max(dims) > max_edge:
            continue
        nx, ny, nz = dims
        flags = random_obstacles((nz, ny, nx), seed=seed * 1000 + c, solid_fraction=frac,
                                 kind="spheres" if c % 4 < 2 else "boxes")
        out.append({"kind": "dense" if c % 2 == 0 else "sparse", "dims": dims, "flags": flags,
                    "tau": tau_c, "u0": u0, "solid_fraction": frac})
    return out


def batch_case_fields(case):
    """Initial (rho, u) of a batch case (2D Taylor-Green of amplitude u0)."""
    return taylor_green_2d(0, u0=case["u0"], dims=case["dims"])


# ------------------------------------------------- reduced accuracy cases
# Small cases of the same shape as each benchmark workload (same layout,
# boundary kinds, relaxation time, start), small enough for the FP64 oracle
# to run them whole.  The library runs each with a bench line's storage,
# schedule and kernel variant; the oracle's velocity at the sampled updated
# voxels is stored once by a script of the oracle package; the comparison
# gives the line's velocity-L2 error against FP64.

ACC_SAMPLES = 2048  # sampled updated voxels per case (per level)


def box_mean(a, r):
    """Mean over r^3 boxes of the last three axes (coarse-level start of a
    multi-resolution case: a coarser level takes the mean of its cubes)."""
    *lead, nz, ny, nx = a.shape
    return a.reshape(*lead, nz // r, r, ny // r, r, nx // r, r).mean(axis=(-5, -3, -1))


def level_fields(rho, u, n_levels):
    """Per-level (rho, u) of a multi-resolution start: level l is the mean of
    the finest field over 2^l cubes."""
    out = [(rho, u)]
    for _ in range(1, n_levels):
        rho, u = box_mean(rho, 2), box_mean(u, 2)
        out.append((rho, u))
    return out


def sample_voxels(mask, n=ACC_SAMPLES, seed=0):
    """Sorted flat indices (x fastest) of up to n voxels drawn without
    replacement from the True entries of mask."""
    idx = np.flatnonzero(np.asarray(mask).ravel())
    if idx.size <= n:
        return idx
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(idx, size=n, replace=False))


def closure_test_network(seed=2025, out_scale=0.02):
    """A fixed 16-64-64-1 network (flat FP32 parameters, the library's order
    W1, b1, W2, b2, W3, b3) whose output varies by ~out_scale over the
    features of a turbulent state: He-initialised layers, the first layer's
    columns scaled by the inverse of each feature's typical magnitude
    (rho - 1 ~ 1e-3, u ~ 3e-2, Pi^neq / (rho c_s^2) ~ 1e-2, its norm and
    trace ~ 1e-2, third moments ~ 1e-3, tau ~ 0.5)."""
    rng = np.random.default_rng(seed)
    typ = np.array([1e-3, 3e-2, 3e-2, 3e-2] + [1e-2] * 6 + [1e-2, 1e-2] + [1e-3] * 3 + [0.5])
    w1 = rng.standard_normal((64, 16)) * np.sqrt(2 / 16) / typ
    return np.concatenate([w1.ravel(), 0.1 * rng.standard_normal(64),
                           rng.standard_normal(64 * 64) * np.sqrt(2 / 64), np.zeros(64),
                           rng.standard_normal(64) * np.sqrt(1 / 64) * out_scale,
                           np.zeros(1)]).astype(np.float32)


def accuracy_cases():
    """Reduced case of every benchmark workload, by name.  Each dict holds
    kind ('dense', 'sparse', 'multires', 'batch'), the inputs both sides
    need (flags and boundary values, level map, start fields per level,
    relaxation time, periodic axes, lattice, closure weights, number of
    steps: coarsest steps on multi-resolution grids) and the sampled voxels
    per level (or per batch case)."""
    cases = {}
    for q in (19, 27):
        flags, bc = cavity(48)
        n = 48
        cases[f"cavity48_q{q}"] = dict(
            kind="dense", q=q, dims=(n, n, n), flags=flags, bc=bc, tau=0.515,
            periodic=(0, 0, 0), steps=100,
            fields=[(np.ones((n, n, n)), np.zeros((3, n, n, n)))],
            what="48^3 lid-driven cavity (the 256^3 workload's boundaries, tau, lid and rest start), 100 steps")
        flags, bc = sphere_channel(dims=(76, 44, 44), radius_channel=19, sphere_center_x=22,
                                   sphere_radius=8, u_in=0.04)
        t = flags & 7
        upd = (t == FLUID) | (t == VELOCITY) | (t == PRESSURE)
        cases[f"sphere_small_q{q}"] = dict(
            kind="sparse", q=q, dims=(76, 44, 44), flags=flags, bc=bc, tau=0.52,
            periodic=(0, 0, 0), steps=100,
            fields=[(np.ones(flags.shape), np.zeros((3,) + flags.shape))],
            what="76x44x44 sphere channel, 8^3 blocks (the 512x256x256 workload's inlet, outlet, "
                 "sphere, tau and rest start), 100 steps")
        lmap = np.array([2, 1, 0, 1], np.uint8).reshape(4, 1, 1)
        rho, u = turbulence(0, seed=7898, u_rms=0.03, dims=(32, 32, 128))
        cases[f"turb3_q{q}"] = dict(
            kind="multires", q=q, dims=(32, 32, 128), n_levels=3, level_map=lmap, flags=None,
            bc=None, tau=0.52, periodic=(1, 1, 1), steps=25, fields=level_fields(rho, u, 3),
            what="3-level periodic map coarse-middle-fine-middle (32x32x128 finest box; the "
                 "256^3 slab map's level jumps, tau_0 and k^-5/3 start), 25 coarsest steps")
    c = dict(cases["turb3_q19"])
    c["theta"] = closure_test_network()
    c["what"] = c["what"] + ", learned closure on levels 1 and 2 (a fixed test network)"
    cases["turb3_closure"] = c
    n = 160
    flags, bc = cavity(n)
    rho, u = np.ones((n, n, n)), np.zeros((3, n, n, n))
    cases["cavity3_160"] = dict(
        kind="multires", q=19, dims=(n, n, n), n_levels=3,
        level_map=multires_cavity_map(n, 3, (1, 1)), flags=flags, bc=bc, tau=0.52,
        periodic=(0, 0, 0), steps=4, fields=level_fields(rho, u, 3),
        what="160^3 3-level lid-driven cavity (the smallest the shell rule allows; the 384^3 "
             "workload's walls, lid, tau_0 and rest start), 4 coarsest steps")
    lmap4 = np.array([3, 2, 1, 0, 1, 2], np.uint8).reshape(6, 1, 1)
    rho, u = turbulence(0, seed=7898, u_rms=0.03, dims=(64, 64, 384))
    cases["mr4_small"] = dict(
        kind="multires", q=19, dims=(64, 64, 384), n_levels=4, level_map=lmap4, flags=None,
        bc=None, tau=0.52, periodic=(1, 1, 1), steps=2, fields=level_fields(rho, u, 4),
        what="4-level periodic map 3-2-1-0-1-2 (64x64x384 finest box; the smallest 4-level "
             "cavity is 448^3), k^-5/3 start, 2 coarsest steps")
    picked = batch_cases(max_edge=64)
    cases["batch_small"] = dict(
        kind="batch", q=19, cases=picked, steps=100, periodic=(1, 1, 1),
        what="the serving batch's cases with every edge <= 64 (two dense, one 8^3 block-sparse; "
             "obstacles, their tau and Taylor-Green start), 100 steps")
    c = dict(cases["batch_small"])
    c["theta"] = closure_test_network()
    c["what"] = c["what"] + ", learned closure on every case (a fixed test network)"
    cases["batch_small_closure"] = c
    return cases


def accuracy_samples(case):
    """Sampled voxels of a case: a list with one array of flat indices per
    level (multires), per batch case (batch), or one (dense, sparse)."""
    if case["kind"] in ("dense", "sparse"):
        t = case["flags"] & 7
        return [sample_voxels((t == FLUID) | (t == VELOCITY) | (t == PRESSURE), seed=1)]
    if case["kind"] == "batch":
        return [sample_voxels((c["flags"] & 7) == FLUID, seed=2 + k)
                for k, c in enumerate(case["cases"])]
    lmap = case["level_map"]
    nx, ny, nz = case["dims"]
    cell = nx // lmap.shape[2]
    out = []
    for lv in range(case["n_levels"]):
        r = cell >> lv
        own = lmap.repeat(r, 0).repeat(r, 1).repeat(r, 2) == lv
        if lv == 0 and case["flags"] is not None:
            t = case["flags"] & 7
            own = own & ((t == FLUID) | (t == VELOCITY) | (t == PRESSURE))
        out.append(sample_voxels(own, seed=10 + lv))
    return out
