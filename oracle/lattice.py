"""D3Q19 lattice for the oracle (FP64).

The paper uses D3Q19 for its dense experiments (Sec. 6, "lattices with 19
(D3Q19) or 27 (D3Q27) directions") and BGK collision (Sec. 6); it does not
list velocities or weights.  Reading adopted (standard D3Q19, Krueger et al.
2016, cited in Sec. 6):

  i = 0           rest
  i = 1..6        (+x) (-x) (+y) (-y) (+z) (-z)
  i = 7..18       (+1,+1,0) (-1,-1,0) (+1,-1,0) (-1,+1,0)
                  (+1,0,+1) (-1,0,-1) (+1,0,-1) (-1,0,+1)
                  (0,+1,+1) (0,-1,-1) (0,+1,-1) (0,-1,+1)

so that every odd index i >= 1 has its opposite at i + 1.
Weights: 1/3 (rest), 1/18 (axis), 1/36 (diagonal); c_s^2 = 1/3.
"""
from fractions import Fraction

import numpy as np

Q = 19

C = np.array(
    [
        (0, 0, 0),
        (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
        (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
    ],
    dtype=np.int64,
)

W_FRAC = [Fraction(1, 3)] + [Fraction(1, 18)] * 6 + [Fraction(1, 36)] * 12
W = np.array([float(w) for w in W_FRAC], dtype=np.float64)

CS2 = 1.0 / 3.0


def _opposite_table():
    """opp[i] = index j with c_j = -c_i, found by search (not by formula)."""
    opp = np.empty(Q, dtype=np.int64)
    for i in range(Q):
        hits = [j for j in range(Q) if np.all(C[j] == -C[i])]
        assert len(hits) == 1
        opp[i] = hits[0]
    return opp


OPP = _opposite_table()

# Outward-normal index used by boundary flags: 0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z.
NORMALS = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
                   dtype=np.int64)


def equilibrium(rho, u):
    """Second-order Maxwell-Boltzmann equilibrium.

    f_i^eq = w_i rho [1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u]

    rho : array of shape S; u : array of shape (3,) + S.
    Returns an array of shape (19,) + S.
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    feq = np.empty((Q,) + rho.shape, dtype=np.float64)
    for i in range(Q):
        cu = C[i, 0] * u[0] + C[i, 1] * u[1] + C[i, 2] * u[2]
        feq[i] = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq)
    return feq


def moments(f):
    """Density and velocity of a population field f of shape (19,) + S."""
    rho = f.sum(axis=0)
    j = np.stack([np.tensordot(C[:, a].astype(np.float64), f, axes=(0, 0)) for a in range(3)])
    return rho, j / rho


def second_moment(f):
    """Pi_ab = sum_i c_ia c_ib f_i, shape (3, 3) + S."""
    Cf = C.astype(np.float64)
    out = np.empty((3, 3) + f.shape[1:], dtype=np.float64)
    for a in range(3):
        for b in range(3):
            out[a, b] = np.tensordot(Cf[:, a] * Cf[:, b], f, axes=(0, 0))
    return out


def regularized_neq(w_pi):
    """f_i^{neq,reg} = 9/2 w_i (c_ia c_ib - delta_ab / 3) Pi^neq_ab.

    The Hermite projection of a non-equilibrium second moment onto the
    populations (regularized LBM, Latt and Chopard 2006/2008, cited in Sec. 1
    and Sec. 6.2).  ``w_pi`` has shape (3, 3) + S.
    """
    Cf = C.astype(np.float64)
    out = np.empty((Q,) + w_pi.shape[2:], dtype=np.float64)
    for i in range(Q):
        acc = 0.0
        for a in range(3):
            for b in range(3):
                qab = Cf[i, a] * Cf[i, b] - (1.0 / 3.0 if a == b else 0.0)
                acc = acc + qab * w_pi[a, b]
        out[i] = 4.5 * W[i] * acc
    return out
