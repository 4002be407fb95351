"""Multi-resolution D3Q19 lattice-Boltzmann step (oracle, FP64).

The paper (Sec. 5; Sec. 6.3) uses one uniform grid per level, refinement
factor 2, and two inter-level operations per time step: explosion (collision
results of a coarse level feed the finer level) and coalescence (streaming
data of the finer level merges into coarse voxels).  It gives no formulas.
Reading implemented here (a volumetric, mass-conserving scheme of the family
of the multi-resolution LBM the paper builds on):

* level 0 is the finest; a level-l voxel is a cube of 2^l finest voxels;
  acoustic scaling dx_l = dt_l = 2^l, so lattice velocities are the same on
  every level and tau_l - 1/2 = (tau_0 - 1/2) / 2^l keeps one physical
  viscosity;
* every region of the box is owned by exactly one level (a level map), with
  2:1 grading;
* one step of a level l > 0 contains two steps of level l-1; the exchange
  across a level jump is defined as level-(l-1) streaming over those two
  substeps in which every level-l voxel is represented by its 8 virtual
  subcells.  Virtual subcells start the coarse step holding the coarse
  post-collision populations C, stream but do not collide;
* explosion (a level-(l-1) voxel p pulls population i from q = p - c_i):
    substep 1: q virtual -> C_i(cell(q));
    substep 2: q virtual -> the value q received in substep 1:
               F0_i(q - c_i) if q - c_i is a level-(l-1) voxel, else
               C_i(cell(q - c_i))            (F0 = fine state at the start);
* coalescence: a level-l voxel X next to level l-1 pulls, for every i, the
  mean over its 8 subcells p of the value p receives in substep 2:
    F1_i(p - c_i) if p - c_i is a level-(l-1) voxel (F1 = fine state after
    substep 1), else the value p - c_i received in substep 1 (as above);
  then X collides with tau_l.
Away from level jumps both rules reduce to plain streaming.  Pure streaming
at the finest resolution is a permutation and averaging keeps the sum of the
8 subcells, so mass and momentum weighted by voxel volume (8^l) are conserved
exactly in a periodic box.  There is no rescaling of non-equilibrium parts
between levels.

Learned closure (optional, not in the paper): on every level l >= 1 each
owned voxel collides with tau_eff = max(tau_l + d_tau, 1/2 + 1e-3), where
d_tau is the closure network (oracle/closure.py) applied to the features of
the populations the voxel pulled this step (after explosion / coalescence)
and tau_l; level 0 keeps tau_0.  The network parameters are used as given
(FP64), so a caller that wants the storage precision of the weights rounds
them first.

Walls and boundaries (the multi-resolution lid-driven cavity of Sec. 6.3,
Table 5).  Reading: they lie on the finest level.  Every map cell touching a
non-periodic box side is owned by level 0, so the coarser levels sit at
least one coarsest block (8 2^(L-1) finest voxels) away from every wall and
no explosion / coalescence trace (at most two finest voxels long) reaches
one.  Level 0 then pulls exactly as the single-resolution oracle does
(halfway bounce-back at non-periodic box sides and solid voxels,
regularized velocity / pressure nodes rebuilt after the collision), with
the pulls whose source a coarser level owns replaced by explosion.

State: f[l] is a (19, nz_l, ny_l, nx_l) array over the whole level-l virtual
box, zero where level l does not own the region (and on level-0 solid
voxels).  Without walls the box is periodic.
"""
import numpy as np

from . import closure as cl
from . import lattice as L
from . import lbm


def tau_of_level(tau0, level):
    return 0.5 + (tau0 - 0.5) / (2 ** level)


def upsample(a):
    """Level l -> level l-1 resolution: every voxel becomes 2x2x2 copies."""
    return a.repeat(2, axis=-1).repeat(2, axis=-2).repeat(2, axis=-3)


def subcell_mean(a):
    """Mean over 2x2x2 subcells by three pairwise means (exact for equal values)."""
    a = 0.5 * (a[..., 0::2] + a[..., 1::2])
    a = 0.5 * (a[..., 0::2, :] + a[..., 1::2, :])
    a = 0.5 * (a[..., 0::2, :, :] + a[..., 1::2, :, :])
    return a


def shift(a, c, k=1):
    """Value at x - k c on a periodic box (last three axes are z, y, x)."""
    return np.roll(a, shift=(k * int(c[2]), k * int(c[1]), k * int(c[0])), axis=(-3, -2, -1))


class MultiRes:
    """Multi-resolution grid: level_map (Mz, My, Mx) gives the owning level of
    every cube of `cell` finest voxels; cell must be a multiple of 2^(L-1)."""

    def __init__(self, level_map, n_levels, cell, tau0, collision="bgk", theta=None,
                 periodic=(True, True, True), flags0=None, bc0=None, q=19):
        """periodic: per axis (x, y, z); flags0: level-0 flag bytes (solid and
        regularized voxels, inside the level-0 region); bc0: (4,) + level-0
        box boundary values of its regularized voxels; q: 19 or 27 (the
        closure is D3Q19 only)."""
        self.lat = L.lattice(q)
        if theta is not None and q != 19:
            raise ValueError("the closure features are those of D3Q19")
        level_map = np.asarray(level_map, dtype=np.int64)
        self.theta = None if theta is None else np.asarray(theta, dtype=np.float64)
        self.periodic = tuple(bool(p) for p in periodic)
        for a, ax in ((0, 2), (1, 1), (2, 0)):     # map axes are (z, y, x)
            if not self.periodic[a]:
                edge = np.concatenate([np.take(level_map, [0], axis=ax).ravel(),
                                       np.take(level_map, [-1], axis=ax).ravel()])
                if np.any(edge != 0):
                    raise ValueError("map cells on a non-periodic side must be level 0")
        assert cell % (2 ** (n_levels - 1)) == 0
        self.L = n_levels
        self.tau0 = tau0
        self.collision = collision
        self.own = []
        for lv in range(n_levels):
            r = cell // (2 ** lv)
            self.own.append(level_map.repeat(r, 0).repeat(r, 1).repeat(r, 2))
        self.f = [np.zeros((self.lat.Q,) + o.shape) for o in self.own]
        self.flags0 = (np.zeros(self.own[0].shape, np.uint8) if flags0 is None
                       else np.asarray(flags0, dtype=np.uint8))
        if np.any((self.flags0 & 7 != 0) & (self.own[0] != 0)):
            raise ValueError("walls and boundary nodes must lie in the level-0 region")
        self.bc0 = None if bc0 is None else np.asarray(bc0, dtype=np.float64)
        t0 = lbm.flag_type(self.flags0)
        self.updated0 = (t0 == lbm.FLUID) | (t0 == lbm.VELOCITY) | (t0 == lbm.PRESSURE)

    def dims(self, level):
        nz, ny, nx = self.own[level].shape
        return nx, ny, nz

    def init_equilibrium(self, level, rho, u):
        feq = self.lat.equilibrium(rho, u)
        mine = self.own[level] == level
        if level == 0:
            mine = mine & self.updated0
        self.f[level] = np.where(mine[None], feq, 0.0)

    def _neighbour_levels(self, lv):
        own = self.own[lv]
        finer = np.zeros(own.shape, bool)
        coarser = np.zeros(own.shape, bool)
        for i in range(1, self.lat.Q):
            nb = shift(own, self.lat.C[i])
            finer |= nb == lv - 1
            coarser |= nb == lv + 1
        return finer, coarser

    def _advance(self, lv, k, f0_self):
        """One step of level lv; k = 1 or 2 is its substep inside the step of
        level lv+1; f0_self = level-lv state at the start of that step."""
        if lv > 0:
            f0_fine = self.f[lv - 1].copy()
            self._advance(lv - 1, 1, f0_fine)
            f1_fine = self.f[lv - 1].copy()
            self._advance(lv - 1, 2, f0_fine)
        S = self.f[lv]
        own = self.own[lv]
        has_finer, _ = self._neighbour_levels(lv)
        g = np.empty_like(S)
        # level 0 pulls as the single-resolution oracle (walls, solids);
        # coarser levels never touch a wall
        base = lbm.stream_with_walls(S, self.flags0, self.periodic) if lv == 0 else None
        for i in range(self.lat.Q):
            c = self.lat.C[i]
            val = base[i] if lv == 0 else shift(S[i], c)
            if lv + 1 < self.L:                       # explosion from level lv+1
                c_up = upsample(self.f[lv + 1][i])
                if k == 1:
                    ex = shift(c_up, c)
                else:
                    ex = np.where(shift(own, c, 2) == lv, shift(f0_self[i], c, 2),
                                  shift(c_up, c, 2))
                val = np.where(shift(own, c) == lv + 1, ex, val)
            if lv > 0:                                # coalescence from level lv-1
                own_f = self.own[lv - 1]
                s_up = upsample(S[i])
                v1 = np.where(shift(own_f, c) == lv - 1, shift(f0_fine[i], c), shift(s_up, c))
                held = np.where(own_f == lv - 1, f1_fine[i], v1)
                coal = subcell_mean(shift(held, c))
                val = np.where(has_finer, coal, val)
            g[i] = val
        tau = tau_of_level(self.tau0, lv)
        if self.theta is not None and lv > 0:
            mine = own == lv
            d_tau, _ = cl.forward(self.theta, cl.features(g[:, mine], tau))
            tau = np.full(own.shape, tau)
            tau[mine] = np.maximum(tau[mine] + d_tau, cl.TAU_MIN)
        with np.errstate(invalid="ignore", divide="ignore"):   # unowned voxels hold zeros
            fnew, _, _ = lbm.collide(g, tau, self.collision)
        mine = own == lv
        if lv == 0:
            types = lbm.flag_type(self.flags0)
            normals = lbm.flag_normal(self.flags0)
            for kind in (lbm.VELOCITY, lbm.PRESSURE):
                for nrm in range(6):
                    sel = (types == kind) & (normals == nrm)
                    if sel.any():
                        fnew[:, sel], _, _ = lbm.regularized_boundary(
                            g[:, sel], nrm, self.bc0[:, sel], kind, tau)
            mine = mine & self.updated0
        self.f[lv] = np.where(mine[None], fnew, 0.0)

    def step(self):
        """One step of the coarsest level (2^(L-1-l) steps of every level l)."""
        self._advance(self.L - 1, 1, None)

    def run(self, n):
        for _ in range(n):
            self.step()

    def conservation(self):
        """(M, Jx, Jy, Jz) weighted by voxel volume 8^l."""
        out = np.zeros(4)
        for lv in range(self.L):
            out += (8.0 ** lv) * lbm.conservation(self.f[lv])
        return out

    def updates_per_step(self):
        return sum(int((self.own[lv] == lv).sum()) * 2 ** (self.L - 1 - lv) for lv in range(self.L))
