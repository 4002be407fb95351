"""Learned relaxation-time closure (oracle, FP64).

Not in the paper: the learned part comes from the benchmark's goal (a per-
voxel MLP that corrects the relaxation time on under-resolved levels of the
multi-resolution solver, trained on data the solver itself generates).
Reading implemented here:

features (16 per voxel, from the pulled populations g and tau of the level)
    rho - 1, u_x, u_y, u_z,
    Pi^neq_{xx,yy,zz,xy,xz,yz} / (rho c_s^2),
    |Pi^neq|_F / (rho c_s^2), tr Pi^neq / (rho c_s^2),
    q_x, q_y, q_z / (rho c_s^2) with q_x = sum_i c_ix (c_iy^2 + c_iz^2) (g_i - f^eq_i)
    (and cyclic), tau
network
    16 -> 64 (ReLU) -> 64 (ReLU) -> 1 (linear) = d_tau
    parameters, flattened in this order: W1 (64 x 16, row j = unit j),
    b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1)  -> 5313 values
collision with the closure
    tau_eff = max(tau + d_tau, 1/2 + 1e-3); `step` is one single-resolution
    time step with it on every fluid voxel (the multi-resolution oracle applies
    it on levels >= 1)
training data
    box-filter a fine periodic run by r^3 (mean of the populations), stream
    the filtered populations one coarse step (the values a coarse voxel
    pulls) and take their features; the target is the least-squares eddy
    viscosity over the 3^3 coarse neighbourhood N(X):
    d_tau = 3 nu_t,  nu_t = - sum_N tau_sgs_dev : S / sum_N 2 rho S : S,
    tau_sgs = mean(rho u u) - rho_bar u_bar u_bar, S from central differences
    of u_bar on the coarse lattice (coarse lattice units), clamped to
    [-(tau_c - 1/2) + 1e-3, 1/2].  (A per-voxel projection is too noisy to
    learn from: the network then explains no variance.)
loss / optimiser
    mean squared error; Adam (beta 0.9, 0.999, eps 1e-8).
training loop (`train`)
    features and targets standardised by their mean and population standard
    deviation over the whole set; a column whose deviation is below 1e-6 of
    its mean's magnitude (or zero) is constant at FP32 precision -- the tau
    feature of a one-level training set -- and keeps scale 1, so rounding
    noise in its deviation never becomes a huge scale in the folded layer; step
    k = 1..K draws its minibatch of B samples by the counter-based SplitMix64
    generator, sample b = splitmix64(seed + (k - 1) B + b) mod n; Adam on the
    standardised problem; the standardisation is folded into the first and
    last layers at the end (`fold_normalisation`).
"""
import numpy as np

from . import lattice as L

N_FEAT = 16
HIDDEN = 64
SIZES = [("W1", (HIDDEN, N_FEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)),
         ("b2", (HIDDEN,)), ("W3", (HIDDEN,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)
TAU_MIN = 0.5 + 1e-3


def unpack(theta):
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def features(g, tau):
    """g: (19, ...) absolute populations; returns (..., 16)."""
    g = np.asarray(g, dtype=np.float64)
    rho = g.sum(axis=0)
    Cf = L.C.astype(np.float64)
    u = np.stack([np.tensordot(Cf[:, a], g, axes=(0, 0)) for a in range(3)]) / rho
    d = g - L.equilibrium(rho, u)
    P = L.second_moment(d)
    s = rho / 3.0
    pxx, pyy, pzz = P[0, 0] / s, P[1, 1] / s, P[2, 2] / s
    pxy, pxz, pyz = P[0, 1] / s, P[0, 2] / s, P[1, 2] / s
    frob = np.sqrt(pxx ** 2 + pyy ** 2 + pzz ** 2 + 2 * (pxy ** 2 + pxz ** 2 + pyz ** 2))
    tr = pxx + pyy + pzz
    q = []
    for a in range(3):
        b, c = [k for k in range(3) if k != a]
        w = Cf[:, a] * (Cf[:, b] ** 2 + Cf[:, c] ** 2)
        q.append(np.tensordot(w, d, axes=(0, 0)) / s)
    tau_f = np.full(rho.shape, float(tau))
    return np.stack([rho - 1.0, u[0], u[1], u[2], pxx, pyy, pzz, pxy, pxz, pyz, frob, tr,
                     q[0], q[1], q[2], tau_f], axis=-1)


def forward(theta, X):
    """X: (n, 16).  Returns (y (n,), cache)."""
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, t):
    """Mean squared error of the network on (X, t) and its gradient (flat)."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dh2 = np.outer(dy, p["W3"])
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def box_filter(a, r):
    """Mean over r^3 boxes of the last three axes."""
    *lead, nz, ny, nx = a.shape
    b = a.reshape(*lead, nz // r, r, ny // r, r, nx // r, r)
    return b.mean(axis=(-5, -3, -1))


def eddy_target(f_fine, r, tau_coarse):
    """Least-squares eddy-viscosity correction of the coarse relaxation time
    for every r^3 box of a fine periodic state (see module docstring)."""
    f = np.asarray(f_fine, dtype=np.float64)
    rho = f.sum(axis=0)
    Cf = L.C.astype(np.float64)
    j = np.stack([np.tensordot(Cf[:, a], f, axes=(0, 0)) for a in range(3)])
    rb = box_filter(rho, r)
    jb = box_filter(j, r)
    ub = jb / rb
    tsgs = np.empty((3, 3) + rb.shape)
    for a in range(3):
        for b in range(3):
            tsgs[a, b] = box_filter(j[a] * j[b] / rho, r) - rb * ub[a] * ub[b]
    grad = np.empty((3, 3) + rb.shape)   # grad[a, b] = d u_b / d x_a
    for a in range(3):
        axis = 2 - a                       # x -> last axis
        for b in range(3):
            grad[a, b] = 0.5 * (np.roll(ub[b], -1, axis=axis) - np.roll(ub[b], 1, axis=axis))
    S = 0.5 * (grad + grad.transpose(1, 0, *range(2, grad.ndim)))
    tr = (tsgs[0, 0] + tsgs[1, 1] + tsgs[2, 2]) / 3.0
    num = 0.0
    den = 0.0
    for a in range(3):
        for b in range(3):
            dev = tsgs[a, b] - (tr if a == b else 0.0)
            num = num + dev * S[a, b]
            den = den + S[a, b] * S[a, b]
    den = 2.0 * rb * den
    num = neighbourhood_sum(num)
    den = neighbourhood_sum(den)
    with np.errstate(invalid="ignore", divide="ignore"):
        nu_t = np.where(den > 0, -num / den, 0.0)
    return np.clip(3.0 * nu_t, -(tau_coarse - 0.5) + 1e-3, 0.5)


def neighbourhood_sum(a):
    """Sum over the periodic 3^3 neighbourhood of every voxel."""
    out = np.zeros_like(a)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out = out + np.roll(a, (dz, dy, dx), axis=(-3, -2, -1))
    return out


def coarse_pulled(f_fine, r):
    """Populations a coarse voxel pulls from the box-filtered fine state."""
    fb = box_filter(f_fine, r)
    out = np.empty_like(fb)
    for i in range(L.Q):
        cx, cy, cz = (int(v) for v in L.C[i])
        out[i] = np.roll(fb[i], shift=(cz, cy, cx), axis=(0, 1, 2))
    return out


def fold_normalisation(theta, mu, sd, y_mean, y_sd):
    """Network trained on (x - mu)/sd -> (y - y_mean)/y_sd, rewritten to take
    raw features and return raw d_tau."""
    p = unpack(theta)
    p["b1"] = p["b1"] - p["W1"] @ (mu / sd)
    p["W1"] = p["W1"] / sd
    p["W3"] = p["W3"] * y_sd
    p["b3"] = p["b3"] * y_sd + y_mean
    return pack(p)


def step(f, flags, tau, theta, collision="bgk", periodic=(False, False, False)):
    """One time step of a single-resolution grid with the closure on every
    fluid voxel: pull with halfway bounce-back (as oracle.lbm.step), features
    of the pulled populations and tau, tau_eff = max(tau + d_tau, 1/2 + 1e-3),
    collision with tau_eff.  Regularized boundary voxels are not supported."""
    from . import lbm
    types = lbm.flag_type(flags)
    if np.any((types == lbm.VELOCITY) | (types == lbm.PRESSURE)):
        raise ValueError("the closure step has no regularized boundaries")
    g = lbm.stream_with_walls(f, flags, periodic)
    fluid = types == lbm.FLUID
    d_tau, _ = forward(theta, features(g[:, fluid], tau))
    tau_eff = np.full(flags.shape, float(tau))
    tau_eff[fluid] = np.maximum(tau + d_tau, TAU_MIN)
    with np.errstate(invalid="ignore", divide="ignore"):
        f_new, _, _ = lbm.collide(g, tau_eff, collision)
    return np.where(fluid[None], f_new, 0.0)


def run(f, flags, tau, theta, n_steps, **kw):
    for _ in range(n_steps):
        f = step(f, flags, tau, theta, **kw)
    return f


# ------------------------------------------------------------ training loop

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(x):
    """SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014) as a function of its 64-bit counter: add the
    golden-ratio increment, then the two xor-shift-multiply rounds and a final
    xor-shift of the published generator."""
    x = (int(x) + _GOLDEN) & _M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _M64
    return x ^ (x >> 31)


def minibatch_indices(seed, step, batch, n):
    """Samples of training step `step` (counted from 1)."""
    c0 = (step - 1) * batch
    return np.array([splitmix64(seed + c0 + b) % n for b in range(batch)], dtype=np.int64)


def standardisation(X, t):
    """(mu, sd, t_mean, t_sd): column means and population standard deviations
    of the features and the target; a constant column (deviation <= 1e-6
    |mean|, or zero) keeps scale 1."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    mu, sd = X.mean(axis=0), X.std(axis=0)
    sd = np.where((sd > 1e-6 * np.abs(mu)) & (sd > 1e-30), sd, 1.0)
    tm, ts = float(t.mean()), float(t.std())
    return mu, sd, tm, (ts if ts > 1e-6 * abs(tm) and ts > 1e-30 else 1.0)


def train(X, t, theta0, steps, batch, lr, seed):
    """Adam on the standardised problem for `steps` SplitMix64 minibatches from
    theta0 (weights of the standardised problem); returns the weights with the
    standardisation folded in (taking raw features, giving raw d_tau) and the
    last minibatch loss (standardised)."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    mu, sd, tm, ts = standardisation(X, t)
    theta = np.asarray(theta0, dtype=np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    loss = None
    for k in range(1, steps + 1):
        idx = minibatch_indices(seed, k, batch, X.shape[0])
        loss, g = loss_and_grad(theta, (X[idx] - mu) / sd, (t[idx] - tm) / ts)
        theta, m, v = adam(theta, g, m, v, k, lr=lr)
    return fold_normalisation(theta, mu, sd, tm, ts), loss
