"""Shared helpers for the GPU parity tests: build a grid through the C ABI,
run the oracle on the same seeded inputs, compare element by element."""
import numpy as np

from oracle import lbm as olbm
from paper_2503_07898_gb300 import workloads as wl

# Tolerance on populations after 100 FP32 steps against the FP64 oracle
# (max relative error over every updated voxel and direction).
F32_RTOL = 1e-5


def bc_list(flags, bc):
    """Per-regularized-voxel boundary values in flag-scan order (x fastest)."""
    t = flags & 7
    sel = (t == wl.VELOCITY) | (t == wl.PRESSURE)
    return np.ascontiguousarray(bc[:, sel].T, dtype=np.float32)


def oracle_bc(flags, bc):
    """The oracle receives the boundary values the GPU receives (FP32 values)."""
    out = np.array(bc, dtype=np.float64, copy=True)
    t = flags & 7
    sel = (t == wl.VELOCITY) | (t == wl.PRESSURE)
    out[:, sel] = bc[:, sel].astype(np.float32).astype(np.float64)
    return out


def make_grid(lbm, kind, flags, bc, tau, collision="bgk", storage="f32",
              periodic=(0, 0, 0), schedule="disaggregated", block_edge=8, lattice=19):
    nz, ny, nx = flags.shape
    phys = lbm.physics(tau, collision, storage, periodic, schedule, lattice=lattice)
    if kind == "dense":
        g = lbm.lbm_grid_create_dense((nx, ny, nz), phys)
        lbm.lbm_set_boundary(g, 0, flags, bc_list(flags, bc) if bc is not None else None)
    else:
        g = lbm.lbm_grid_create_sparse((nx, ny, nz), block_edge, flags, phys)
        lbm.lbm_set_boundary(g, 0, None, bc_list(flags, bc) if bc is not None else None)
    return g


def run_oracle(flags, bc, rho, u, tau, steps, collision="bgk", periodic=(0, 0, 0), q=19):
    f = olbm.init_equilibrium(rho, u, flags, q=q)
    obc = oracle_bc(flags, bc) if bc is not None else None
    for _ in range(steps):
        f = olbm.step(f, flags, tau, collision=collision, periodic=periodic, bc=obc)
    return f


def updated_mask(flags):
    t = flags & 7
    return (t == 0) | (t == 2) | (t == 3)


def max_rel_err(f_gpu, f_ref, flags):
    m = updated_mask(flags)
    a = f_gpu[:, m]
    b = f_ref[:, m]
    assert np.all(np.isfinite(a)), "non-finite GPU populations on updated voxels"
    return float(np.max(np.abs(a - b) / np.abs(b)))


def velocity_l2(u_gpu, u_ref, flags):
    m = updated_mask(flags)
    d = (u_gpu[:, m] - u_ref[:, m]) ** 2
    return float(np.sqrt(d.sum() / (u_ref[:, m] ** 2).sum()))


def oracle_window(flags, bc, rho, u, center_zyx, steps, tau, collision="bgk"):
    """Oracle populations at one voxel after `steps` steps, computed on the
    sub-box of half-width steps+1 around it (the update has a light cone of
    one voxel per step, so the cut sides cannot reach the centre).  Axes are
    non-periodic; a window side that reaches the real box side keeps the
    real wall."""
    sl = []
    cen = []
    for a, c in enumerate(center_zyx):
        lo = max(0, c - steps - 1)
        hi = min(flags.shape[a], c + steps + 2)
        sl.append(slice(lo, hi))
        cen.append(c - lo)
    sl = tuple(sl)
    fl = np.ascontiguousarray(flags[sl])
    sub_bc = np.ascontiguousarray(bc[(slice(None),) + sl]) if bc is not None else None
    f = run_oracle(fl, sub_bc, rho[sl], u[(slice(None),) + sl], tau, steps, collision)
    return f[(slice(None),) + tuple(cen)]
