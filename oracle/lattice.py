"""D3Q19 and D3Q27 lattices for the oracle (FP64).

The paper uses D3Q19 for its dense experiments and D3Q27 for the
block-sparse register-pressure and strong-scaling studies (Sec. 6); it lists
neither velocities nor weights.  Reading adopted (the standard sets, Krueger
et al. 2016, cited in Sec. 6), ordered so that every odd index i >= 1 has its
opposite at i + 1:

  i = 0           rest
  i = 1..6        (+x) (-x) (+y) (-y) (+z) (-z)
  i = 7..18       (+1,+1,0) (-1,-1,0) (+1,-1,0) (-1,+1,0)
                  (+1,0,+1) (-1,0,-1) (+1,0,-1) (-1,0,+1)
                  (0,+1,+1) (0,-1,-1) (0,+1,-1) (0,-1,+1)
  i = 19..26      (D3Q27 only) (+1,+1,+1) (-1,-1,-1) (+1,+1,-1) (-1,-1,+1)
                  (+1,-1,+1) (-1,+1,-1) (-1,+1,+1) (+1,-1,-1)

Weights: D3Q19 1/3 (rest), 1/18 (axis), 1/36 (edge); D3Q27 8/27, 2/27,
1/54 (edge), 1/216 (corner); c_s^2 = 1/3 for both.  The module-level names
(Q, C, W, OPP, equilibrium, ...) are those of D3Q19; `lattice(q)` returns
either set, and functions taking populations infer it from their length.
"""
from fractions import Fraction

import numpy as np

_C19 = [
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
]
_C27 = _C19 + [
    (1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1),
    (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1),
]
_W19 = [Fraction(1, 3)] + [Fraction(1, 18)] * 6 + [Fraction(1, 36)] * 12
_W27 = [Fraction(8, 27)] + [Fraction(2, 27)] * 6 + [Fraction(1, 54)] * 12 + [Fraction(1, 216)] * 8


def _opposite_table(C):
    """opp[i] = index j with c_j = -c_i, found by search (not by formula)."""
    q = len(C)
    opp = np.empty(q, dtype=np.int64)
    for i in range(q):
        hits = [j for j in range(q) if np.all(C[j] == -C[i])]
        assert len(hits) == 1
        opp[i] = hits[0]
    return opp


class Lattice:
    """One velocity set: Q, C (Q x 3), W, W_FRAC, OPP and the moment
    operations on populations of shape (Q,) + S."""

    def __init__(self, velocities, weights):
        self.Q = len(velocities)
        self.C = np.array(velocities, dtype=np.int64)
        self.W_FRAC = list(weights)
        self.W = np.array([float(w) for w in weights], dtype=np.float64)
        self.OPP = _opposite_table(self.C)

    def equilibrium(self, rho, u):
        """f_i^eq = w_i rho [1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u]; rho of
        shape S, u of shape (3,) + S; returns (Q,) + S."""
        rho = np.asarray(rho, dtype=np.float64)
        u = np.asarray(u, dtype=np.float64)
        usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
        feq = np.empty((self.Q,) + rho.shape, dtype=np.float64)
        for i in range(self.Q):
            cu = self.C[i, 0] * u[0] + self.C[i, 1] * u[1] + self.C[i, 2] * u[2]
            feq[i] = self.W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq)
        return feq

    def moments(self, f):
        rho = f.sum(axis=0)
        j = np.stack([np.tensordot(self.C[:, a].astype(np.float64), f, axes=(0, 0))
                      for a in range(3)])
        return rho, j / rho

    def second_moment(self, f):
        """Pi_ab = sum_i c_ia c_ib f_i, shape (3, 3) + S."""
        Cf = self.C.astype(np.float64)
        out = np.empty((3, 3) + f.shape[1:], dtype=np.float64)
        for a in range(3):
            for b in range(3):
                out[a, b] = np.tensordot(Cf[:, a] * Cf[:, b], f, axes=(0, 0))
        return out

    def regularized_neq(self, w_pi):
        """f_i^{neq,reg} = 9/2 w_i (c_ia c_ib - delta_ab / 3) Pi^neq_ab: the
        Hermite projection of a non-equilibrium second moment onto the
        populations (regularized LBM, Latt and Chopard, cited in Sec. 1 and
        Sec. 6.2).  ``w_pi`` has shape (3, 3) + S."""
        Cf = self.C.astype(np.float64)
        out = np.empty((self.Q,) + w_pi.shape[2:], dtype=np.float64)
        for i in range(self.Q):
            acc = 0.0
            for a in range(3):
                for b in range(3):
                    qab = Cf[i, a] * Cf[i, b] - (1.0 / 3.0 if a == b else 0.0)
                    acc = acc + qab * w_pi[a, b]
            out[i] = 4.5 * self.W[i] * acc
        return out


D3Q19 = Lattice(_C19, _W19)
D3Q27 = Lattice(_C27, _W27)


def lattice(q):
    return {19: D3Q19, 27: D3Q27}[int(q)]


Q, C, W, W_FRAC, OPP = D3Q19.Q, D3Q19.C, D3Q19.W, D3Q19.W_FRAC, D3Q19.OPP

CS2 = 1.0 / 3.0


# Outward-normal index used by boundary flags: 0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z.
NORMALS = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
                   dtype=np.int64)


def equilibrium(rho, u, q=19):
    """Equilibrium of lattice(q) (D3Q19 by default), shape (q,) + S."""
    return lattice(q).equilibrium(rho, u)


def moments(f):
    """Density and velocity of a population field of shape (Q,) + S."""
    return lattice(f.shape[0]).moments(f)


def second_moment(f):
    """Pi_ab = sum_i c_ia c_ib f_i for populations of shape (Q,) + S."""
    return lattice(f.shape[0]).second_moment(f)


def regularized_neq(w_pi, q=19):
    """Regularized non-equilibrium populations of lattice(q) (shape (q,) + S)."""
    return lattice(q).regularized_neq(w_pi)
