"""Plain FP64 D3Q19 / D3Q27 lattice-Boltzmann step on a virtual box (oracle).

State
  f    : float64 array (Q, nz, ny, nx), Q = 19 or 27 (the lattice is read
         from this length), the stored post-collision
         populations f* of every voxel (x fastest).  Voxels that are not
         updated (solid, not in domain) hold 0.
  flags: uint8 array (nz, ny, nx).  Bits 0-2 = type
           0 fluid, 1 solid (bounce-back), 2 regularized velocity node,
           3 regularized pressure node, 7 not in domain;
         bits 3-5 = outward normal index (0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z),
         read for types 2 and 3 only.
  bc   : float64 array (4, nz, ny, nx) = (ux, uy, uz, rho) prescribed at
         regularized nodes (velocity nodes use u, pressure nodes use rho).

One step (pull scheme; the paper fuses collision, streaming and boundary
handling into one update per voxel, Sec. 6):

  1. stream      g_i(x) = f*_i(x - c_i)
  2. walls       if x - c_i is solid, not in domain, or outside a
                 non-periodic box side: halfway bounce-back
                 g_i(x) = f*_opp(i)(x)      (bounce-back, Sec. 6.2)
  3. boundaries  at a regularized node with outward normal n the unknown
                 set U = {i : c_i.n < 0} is rebuilt instead of bounced back
                 (regularized boundaries, Sec. 6.2, Latt et al. 2008):
                   velocity node: rho = (S0 + 2 S+) / (1 + u_b.n)
                   pressure node: u   = ((S0 + 2 S+) / rho_b - 1) n
                   (S0 = sum over c_i.n = 0, S+ = sum over c_i.n > 0)
                   g_i = f^eq_i + (g_opp(i) - f^eq_opp(i))       for i in U
                   Pi^neq = sum_i c_i c_i (g_i - f^eq_i)
                   f* = f^eq + (1 - 1/tau) * 9/2 w_i Q_i : Pi^neq
  4. collide     BGK: f* = g - (g - f^eq(rho, u)) / tau          (Sec. 6)
                 REG: f* = f^eq + (1 - 1/tau) * 9/2 w_i Q_i : Pi^neq(g)
  5. store       f* of updated voxels; 0 elsewhere.

Readings (the paper writes none of these formulas): velocity set, weights,
equilibrium and the regularized boundary follow the references the paper
cites (Krueger et al. 2016; Latt et al. 2008).  At a regularized node the
collision of the reconstructed populations is written directly in its
regularized form (for a regularized input BGK and REG coincide).  The
unknown set follows the node's single normal; every other missing source is
bounced back first (edges and corners).
"""
import numpy as np

from . import lattice as L

FLUID, SOLID, VELOCITY, PRESSURE, OUTSIDE = 0, 1, 2, 3, 7


def flag_type(flags):
    return flags & 7


def flag_normal(flags):
    return (flags >> 3) & 7


def make_flag(kind, normal=0):
    return np.uint8((kind & 7) | ((normal & 7) << 3))


def _shift(a, cz, cy, cx):
    """Value at (z - cz, y - cy, x - cx), periodic wrap (np.roll semantics)."""
    return np.roll(a, shift=(cz, cy, cx), axis=(0, 1, 2))


def _source_outside(shape, c, periodic):
    """True where x - c leaves the box across a non-periodic side."""
    nz, ny, nx = shape
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    out = np.zeros(shape, dtype=bool)
    for coord, n, ci, per in ((x, nx, c[0], periodic[0]), (y, ny, c[1], periodic[1]),
                              (z, nz, c[2], periodic[2])):
        if per:
            continue
        s = coord - ci
        out = out | (s < 0) | (s >= n)
    return out


def stream_with_walls(f, flags, periodic):
    """Steps 1-2: pulled populations g with halfway bounce-back at walls.

    Returns g of shape (Q,) + box (Q = 19 or 27, from f).  Rows of U at
    regularized nodes are still the pulled (or bounced) values;
    ``regularized_boundary`` replaces them.
    """
    lat = L.lattice(f.shape[0])
    types = flag_type(flags)
    g = np.empty_like(f)
    for i in range(lat.Q):
        cx, cy, cz = (int(v) for v in lat.C[i])
        src_val = _shift(f[i], cz, cy, cx)
        src_type = _shift(types, cz, cy, cx)
        wall = (src_type == SOLID) | (src_type == OUTSIDE)
        wall = wall | _source_outside(flags.shape, (cx, cy, cz), periodic)
        g[i] = np.where(wall, f[lat.OPP[i]], src_val)
    return g


def regularized_boundary(g_node, normal, bc_node, kind, tau):
    """Step 3 for a set of nodes sharing one normal.

    g_node : (Q, n) pulled populations; normal: int 0..5; bc_node: (4, n);
    kind   : VELOCITY or PRESSURE.
    Returns (f_star (Q, n), rho (n,), u (3, n)).
    """
    lat = L.lattice(g_node.shape[0])
    nvec = L.NORMALS[normal]
    cn = lat.C @ nvec                    # c_i . n for every i
    k0 = np.flatnonzero(cn == 0)
    kp = np.flatnonzero(cn > 0)
    unknown = np.flatnonzero(cn < 0)
    s = g_node[k0].sum(axis=0) + 2.0 * g_node[kp].sum(axis=0)
    if kind == VELOCITY:
        u = bc_node[0:3].copy()
        un = nvec[0] * u[0] + nvec[1] * u[1] + nvec[2] * u[2]
        rho = s / (1.0 + un)
    else:
        rho = bc_node[3].copy()
        un = s / rho - 1.0
        u = np.stack([un * nvec[0], un * nvec[1], un * nvec[2]]).astype(np.float64)
    feq = lat.equilibrium(rho, u)
    g = g_node.copy()
    for i in unknown:
        j = lat.OPP[i]
        g[i] = feq[i] + (g[j] - feq[j])
    pi_neq = lat.second_moment(g - feq)
    fneq = lat.regularized_neq(pi_neq)
    f_star = feq + (1.0 - 1.0 / tau) * fneq
    return f_star, rho, u


def collide(g, tau, collision="bgk", force=None):
    """Step 4 on pulled populations g (Q,) + S.  Returns (f*, rho, u).

    ``force`` (3 floats) adds a constant body force with Guo's scheme
    (velocity shifted by F/2, source (1 - 1/(2 tau)) w_i [3(c_i - u) +
    9 (c_i.u) c_i].F); it exists only for the Poiseuille pin.
    """
    lat = L.lattice(g.shape[0])
    rho = g.sum(axis=0)
    Cf = lat.C.astype(np.float64)
    j = np.stack([np.tensordot(Cf[:, a], g, axes=(0, 0)) for a in range(3)])
    if force is not None:
        j = j + 0.5 * np.asarray(force, dtype=np.float64).reshape((3,) + (1,) * rho.ndim)
    u = j / rho
    feq = lat.equilibrium(rho, u)
    if collision == "bgk":
        f_star = g - (g - feq) / tau
    elif collision == "reg":
        f_star = feq + (1.0 - 1.0 / tau) * lat.regularized_neq(lat.second_moment(g - feq))
    else:
        raise ValueError(collision)
    if force is not None:
        F = np.asarray(force, dtype=np.float64)
        for i in range(lat.Q):
            cu = Cf[i, 0] * u[0] + Cf[i, 1] * u[1] + Cf[i, 2] * u[2]
            src = 0.0
            for a in range(3):
                src = src + (3.0 * (Cf[i, a] - u[a]) + 9.0 * cu * Cf[i, a]) * F[a]
            f_star[i] = f_star[i] + (1.0 - 0.5 / tau) * lat.W[i] * src
    return f_star, rho, u


def step(f, flags, tau, collision="bgk", periodic=(False, False, False), bc=None,
         force=None, return_macro=False):
    """One full time step on the virtual box; returns the new f* (and rho, u)."""
    types = flag_type(flags)
    g = stream_with_walls(f, flags, periodic)
    f_new, rho, u = collide(g, tau, collision, force)
    reg = (types == VELOCITY) | (types == PRESSURE)
    if reg.any():
        if bc is None:
            raise ValueError("regularized nodes need bc values")
        normals = flag_normal(flags)
        for kind in (VELOCITY, PRESSURE):
            for nrm in range(6):
                sel = (types == kind) & (normals == nrm)
                if not sel.any():
                    continue
                fs, r, uu = regularized_boundary(g[:, sel], nrm, bc[:, sel], kind, tau)
                f_new[:, sel] = fs
                rho[sel] = r
                u[:, sel] = uu
    updated = (types == FLUID) | reg
    f_new = np.where(updated[None], f_new, 0.0)
    if return_macro:
        return f_new, rho, u
    return f_new


def run(f, flags, tau, n_steps, **kw):
    for _ in range(n_steps):
        f = step(f, flags, tau, **kw)
    return f


def init_equilibrium(rho, u, flags=None, q=19):
    """Initial state f* = f^eq(rho, u) of lattice(q) in FP64 (0 on voxels
    not updated)."""
    f = L.equilibrium(rho, u, q)
    if flags is not None:
        t = flag_type(flags)
        upd = (t == FLUID) | (t == VELOCITY) | (t == PRESSURE)
        f = np.where(upd[None], f, 0.0)
    return f


def state_moments(f, flags=None):
    """Density and velocity of the stored state; NaN on voxels not updated."""
    rho = f.sum(axis=0)
    Cf = L.lattice(f.shape[0]).C.astype(np.float64)
    j = np.stack([np.tensordot(Cf[:, a], f, axes=(0, 0)) for a in range(3)])
    with np.errstate(invalid="ignore", divide="ignore"):
        u = j / rho
    if flags is not None:
        t = flag_type(flags)
        upd = (t == FLUID) | (t == VELOCITY) | (t == PRESSURE)
        rho = np.where(upd, rho, np.nan)
        u = np.where(upd[None], u, np.nan)
    return rho, u


def conservation(f, flags=None):
    """(M, Jx, Jy, Jz) = sums of f*_i and f*_i c_i over updated voxels."""
    if flags is not None:
        t = flag_type(flags)
        upd = (t == FLUID) | (t == VELOCITY) | (t == PRESSURE)
        f = np.where(upd[None], f, 0.0)
    Cf = L.lattice(f.shape[0]).C.astype(np.float64)
    m = f.sum()
    j = [float(np.tensordot(Cf[:, a], f, axes=(0, 0)).sum()) for a in range(3)]
    return np.array([m] + j)


# ---------------------------------------------------------------- closed forms

def tgv_energy_ratio(tau, k, t):
    """Kinetic-energy ratio E(t)/E(0) of the 2D Taylor-Green vortex.

    u = u0 exp(-2 nu k^2 t) (...) is an exact incompressible Navier-Stokes
    solution for wavenumber k in x and y; E is quadratic in u, so
    E(t)/E(0) = exp(-4 nu k^2 t) with nu = (tau - 1/2) / 3 in lattice units.
    """
    nu = (tau - 0.5) / 3.0
    return float(np.exp(-4.0 * nu * k * k * t))


def poiseuille_profile(g, nu, h):
    """Steady plane-channel profile for walls at y = -1/2 and y = h - 1/2.

    u(y) = g / (2 nu) (y + 1/2)(h - 1/2 - y) for a body force g along x.
    """
    y = np.arange(h, dtype=np.float64)
    return g / (2.0 * nu) * (y + 0.5) * (h - 0.5 - y)
