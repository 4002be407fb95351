"""Pins of the learned-closure oracle (oracle/closure.py): the network's
gradient against finite differences, a hand-built network, Adam's first step,
the features on inputs whose moments are known, and the training target's
invariances; the single-grid closure step against plain steps it must
reduce to."""
import numpy as np
import pytest

from oracle import closure as cl
from oracle import lattice as L
from oracle import lbm as olbm
from paper_2503_07898_gb300 import workloads as wl


def random_theta(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(cl.N_PARAMS) * scale


def test_parameter_count():
    assert cl.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1 == 5313


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = random_theta(2)
    X = rng.standard_normal((37, 16))
    t = rng.standard_normal(37)
    _, g = cl.loss_and_grad(theta, X, t)
    h = 1e-6
    for k in list(range(0, 1024, 97)) + [1024 + 5, 1088 + 700, 5184 + 3, 5248 + 10, 5312]:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (cl.loss_and_grad(theta + e, X, t)[0] - cl.loss_and_grad(theta - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_hand_built_network():
    """W1 copies the 16 features into units 0..15, W2 is the identity, W3 sums:
    the output is the sum of the positive parts of the features (+ b3)."""
    p = {"W1": np.zeros((64, 16)), "b1": np.zeros(64), "W2": np.eye(64), "b2": np.zeros(64),
         "W3": np.ones(64), "b3": np.array([0.25])}
    p["W1"][:16] = np.eye(16)
    X = np.random.default_rng(3).standard_normal((9, 16))
    y, _ = cl.forward(cl.pack(p), X)
    assert np.allclose(y, np.maximum(X, 0).sum(axis=1) + 0.25, atol=1e-14)


def test_flat_parameter_layout():
    """The flat parameter vector is, in order, W1 (64 x 16, row j = unit j),
    b1 (64), W2 (64 x 64, row j = unit j), b2 (64), W3 (64), b3 (1): the
    layout the library's kernels read.  Built here by offset, without pack:
    unit 5 of layer 1 reads feature 2, unit 7 of layer 2 reads unit 5 with
    bias 0.01, the other layer-2 units have negative biases, and the output
    is 2 h2_7 + 0.1 = 2 max(x_2, 0) + 0.12."""
    H, F = 64, 16
    o_W1, o_b1 = 0, H * F
    o_W2 = o_b1 + H
    o_b2 = o_W2 + H * H
    o_W3 = o_b2 + H
    o_b3 = o_W3 + H
    assert o_b3 + 1 == cl.N_PARAMS
    theta = np.zeros(cl.N_PARAMS)
    theta[o_W1 + 5 * F + 2] = 1.0
    theta[o_W2 + 7 * H + 5] = 1.0
    theta[o_b2:o_b2 + H] = -0.01 * np.arange(1, H + 1)
    theta[o_b2 + 7] = 0.01
    theta[o_W3 + 7] = 2.0
    theta[o_b3] = 0.1
    X = np.random.default_rng(46).standard_normal((11, F))
    y, _ = cl.forward(theta, X)
    assert np.allclose(y, 2 * np.maximum(X[:, 2], 0) + 0.12, rtol=0, atol=1e-15)


def test_adam_first_step_moves_each_parameter_by_lr():
    theta = random_theta(4)
    grad = np.random.default_rng(5).standard_normal(cl.N_PARAMS)
    new, m, v = cl.adam(theta, grad, np.zeros_like(theta), np.zeros_like(theta), 1, lr=1e-3)
    # bias-corrected moments are g and g^2 after one step: the update is
    # -lr g / (|g| + eps), i.e. -lr sign(g) away from tiny gradients
    assert np.allclose(new - theta, -1e-3 * grad / (np.abs(grad) + 1e-8), rtol=1e-9, atol=0)
    big = np.abs(grad) > 1e-2
    assert np.allclose((new - theta)[big], -1e-3 * np.sign(grad[big]), rtol=1e-5)


def test_features_of_known_populations():
    rho, u = np.array([1.03, 0.98]), np.array([[0.02, -0.01], [0.0, 0.03], [-0.015, 0.005]])
    feq = L.equilibrium(rho, u)
    F = cl.features(feq, 0.51)
    assert np.allclose(F[:, 0], rho - 1, atol=1e-15)
    assert np.allclose(F[:, 1:4], u.T, atol=1e-15)
    assert np.allclose(F[:, 4:15], 0, atol=1e-14)
    assert np.allclose(F[:, 15], 0.51)
    # regularized non-equilibrium with a known Pi: normalised Pi, its norm and trace
    Pi = np.array([[1e-3, 2e-4, -3e-4], [2e-4, -5e-4, 1e-4], [-3e-4, 1e-4, 2e-4]])
    g = feq + L.regularized_neq(np.broadcast_to(Pi[:, :, None], (3, 3, 2)))
    F = cl.features(g, 0.51)
    s = rho / 3
    want = np.array([Pi[0, 0], Pi[1, 1], Pi[2, 2], Pi[0, 1], Pi[0, 2], Pi[1, 2]])
    assert np.allclose(F[:, 4:10], want[None] / s[:, None], rtol=1e-9, atol=0)
    assert np.allclose(F[:, 11], np.trace(Pi) / s, rtol=1e-9)
    assert np.allclose(F[:, 10], np.sqrt((Pi * Pi).sum()) / s, rtol=1e-9)
    # one perturbed population: third-order features pick c_x (c_y^2 + c_z^2) etc.
    i = 7                                                    # (+1, +1, 0)
    g = feq.copy()
    g[i] += 1e-4 * np.array([1.0, 1.0])
    F = cl.features(g, 0.51)
    # the equilibrium is re-evaluated at the perturbed moments; compare with the
    # features computed from the definition directly
    r2 = g.sum(0)
    u2 = np.stack([(L.C[:, a, None] * g).sum(0) for a in range(3)]) / r2
    d = g - L.equilibrium(r2, u2)
    qx = (L.C[:, 0] * (L.C[:, 1] ** 2 + L.C[:, 2] ** 2)) @ d / (r2 / 3)
    assert np.allclose(F[:, 12], qx, rtol=1e-10)


def test_feature_moments_through_closed_equilibrium_moments():
    """The closure kernels form the non-equilibrium moments of the features
    from the moments of the shifted populations s = f - w minus the
    equilibrium's closed-form moments: sum c_a c_b (f^eq - w) = (rho - 1)/3
    delta_ab + rho u_a u_b and sum c_a (|c|^2 - c_a^2) (f^eq - w) = 2/3 rho
    u_a.  On random populations that reading gives the oracle's features
    (which subtract the equilibrium population by population)."""
    rng = np.random.default_rng(61)
    rho = 1.0 + 0.02 * rng.standard_normal(50)
    u = 0.05 * rng.standard_normal((3, 50))
    g = L.equilibrium(rho, u) + 1e-3 * rng.standard_normal((19, 50))
    F = cl.features(g, 0.53)
    s = g - L.W[:, None]
    C = L.C.astype(float)
    r = g.sum(0)
    j = C.T @ g
    uu = j / r
    P = np.einsum("ia,ib,iv->abv", C, C, s) - (r - 1) / 3 * np.eye(3)[:, :, None] \
        - r * uu[:, None, :] * uu[None, :, :]
    k = 3 / r
    want = np.stack([P[0, 0], P[1, 1], P[2, 2], P[0, 1], P[0, 2], P[1, 2]]) * k
    assert np.allclose(F[:, 4:10].T, want, rtol=0, atol=1e-13)
    for a in range(3):
        b, c = [m for m in range(3) if m != a]
        q = (C[:, a] * (C[:, b] ** 2 + C[:, c] ** 2)) @ s - 2 / 3 * j[a]
        assert np.allclose(F[:, 12 + a], q * k, rtol=0, atol=1e-13)


def _fine_feq(u, rho=None):
    shape = u.shape[1:]
    rho = np.ones(shape) if rho is None else rho
    return L.equilibrium(rho, u)


def test_eddy_target_zero_for_box_uniform_fields():
    rng = np.random.default_rng(6)
    uc = 0.01 * rng.standard_normal((3, 4, 4, 4))
    u = uc.repeat(2, 1).repeat(2, 2).repeat(2, 3)          # constant in every 2^3 box
    t = cl.eddy_target(_fine_feq(u), 2, 0.51)
    assert np.allclose(t, 0.0, atol=1e-15)
    # a varying density does not create sub-filter stress when u is box-uniform
    rho = 1.0 + 0.02 * rng.random((8, 8, 8))
    t = cl.eddy_target(_fine_feq(u, rho), 2, 0.51)
    assert np.allclose(t, 0.0, atol=1e-12)


def test_eddy_target_galilean_invariance_and_linearity():
    """With rho = 1 the target is unchanged by a uniform velocity and scales
    linearly with the velocity fluctuation amplitude (tau_sgs ~ A^2, S ~ A)."""
    _, u = wl.turbulence(16, seed=8, u_rms=1e-3, kmax=6)
    t1 = cl.eddy_target(_fine_feq(u), 2, 0.51)
    shift = np.array([0.01, -0.02, 0.005])[:, None, None, None]
    t2 = cl.eddy_target(_fine_feq(u + shift), 2, 0.51)
    t3 = cl.eddy_target(_fine_feq(2 * u), 2, 0.51)
    inner = (t1 > -0.009) & (t1 < 0.49) & (t3 > -0.009) & (t3 < 0.49)   # unclamped
    assert inner.mean() > 0.9
    assert np.allclose(t1, t2, atol=1e-9)
    assert np.allclose(t3[inner], 2 * t1[inner], rtol=1e-6, atol=1e-12)


def test_fold_normalisation_is_exact():
    rng = np.random.default_rng(9)
    theta = random_theta(10)
    X = rng.standard_normal((11, 16)) * 3 + 1
    mu, sd = X.mean(0), X.std(0)
    y_n, _ = cl.forward(theta, (X - mu) / sd)
    folded = cl.fold_normalisation(theta, mu, sd, 0.3, 2.0)
    y, _ = cl.forward(folded, X)
    assert np.allclose(y, y_n * 2.0 + 0.3, rtol=1e-12, atol=1e-12)


def test_coarse_pulled_uniform_flow_is_stationary():
    rho = np.full((8, 8, 8), 1.01)
    u = np.zeros((3, 8, 8, 8))
    u[:] = np.array([0.02, 0.0, -0.01])[:, None, None, None]
    f = L.equilibrium(rho, u)
    assert np.allclose(cl.coarse_pulled(f, 2), L.equilibrium(rho[:4, :4, :4], u[:, :4, :4, :4]),
                       atol=1e-15)


# ------------------------------------------------- single-grid closure step

def _obstacle_box(seed, shape=(10, 9, 12)):
    flags = wl.random_obstacles(shape, seed=seed, solid_fraction=0.1)
    rho, u = wl.random_fields(shape, seed=seed + 1)
    return flags, olbm.init_equilibrium(rho, u, flags)


def _const_net(b3):
    return np.concatenate([np.zeros(cl.N_PARAMS - 1), [b3]])


@pytest.mark.parametrize("b3", [0.0, 0.04, -0.05, -1.0])
def test_closure_step_with_constant_network_is_plain_step(b3):
    """Constant output b3: the plain oracle step at max(tau + b3, 1/2 + 1e-3),
    walls, obstacles and periodic axes included."""
    flags, f0 = _obstacle_box(200)
    per = (True, False, True)
    got = cl.run(f0, flags, 0.58, _const_net(b3), 3, periodic=per)
    ref = olbm.run(f0, flags, max(0.58 + b3, 0.5 + 1e-3), 3, periodic=per)
    assert np.max(np.abs(got - ref)) < 1e-15


def test_closure_step_feeds_tau_and_pulled_moments():
    """d_tau = relu(relu(feature 15)) = tau relaxes with 2 tau; a network
    reading u_x (feature 1) gives tau_eff = tau + 2 relu(u_x) of the pulled
    populations, checked voxel by voxel against a hand evaluation."""
    flags, f0 = _obstacle_box(201)
    p = cl.unpack(_const_net(0.0))
    p["W1"][0, 15] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0] = 1.0
    got = cl.step(f0, flags, 0.6, cl.pack(p), periodic=(True, True, True))
    ref = olbm.step(f0, flags, 1.2, periodic=(True, True, True))
    assert np.max(np.abs(got - ref)) < 1e-15
    p = cl.unpack(_const_net(0.0))
    p["W1"][0, 1] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0] = 2.0
    got = cl.step(f0, flags, 0.6, cl.pack(p), periodic=(True, True, True))
    g = olbm.stream_with_walls(f0, flags, (True, True, True))
    fluid = olbm.flag_type(flags) == olbm.FLUID
    for z, y, x in zip(*np.nonzero(fluid)):
        gv = g[:, z, y, x]
        ux = float(L.C[:, 0] @ gv) / gv.sum()
        fv, _, _ = olbm.collide(gv, 0.6 + 2 * max(ux, 0.0))
        assert np.max(np.abs(got[:, z, y, x] - fv)) < 1e-15


def test_closure_step_conserves_mass_in_a_walled_box():
    flags, f0 = _obstacle_box(202)
    rng = np.random.default_rng(203)
    th = rng.standard_normal(cl.N_PARAMS) * 0.05
    f1 = cl.run(f0, flags, 0.6, th, 5, periodic=(False, False, False))
    m0, m1 = f0.sum(), f1.sum()
    assert abs(m1 - m0) / m0 < 1e-13


# ------------------------------------- filter, coarse pull and target pins
# Each case below is built so that its answer follows by hand from the
# definitions (box mean over r^3, pull g_i(X) = f_i(X - c_i), eddy viscosity
# nu_t = -<tau_sgs_dev : S> / <2 rho S : S>, d_tau = 3 nu_t in coarse lattice
# units), so a reversed difference, a flipped sign, a dropped factor or a
# transposed axis in the oracle fails one of them.

def test_box_filter_brute_force_on_distinct_values():
    """Mean over every r^3 box of a non-cubic array with distinct values,
    against explicit slicing (a transposed reshape mixes boxes)."""
    rng = np.random.default_rng(31)
    a = rng.standard_normal((2, 4, 6, 8))          # (lead, nz, ny, nx)
    got = cl.box_filter(a, 2)
    assert got.shape == (2, 2, 3, 4)
    for l in range(2):
        for Z in range(2):
            for Y in range(3):
                for X in range(4):
                    box = a[l, 2 * Z:2 * Z + 2, 2 * Y:2 * Y + 2, 2 * X:2 * X + 2]
                    assert abs(got[l, Z, Y, X] - box.mean()) < 1e-15
    # r = 3 on a 2^3-distinct pattern: every box holds the same 27 values once
    b = np.arange(6 * 9 * 3, dtype=np.float64).reshape(6, 9, 3)
    got = cl.box_filter(b, 3)
    for Z in range(2):
        for Y in range(3):
            assert got[Z, Y, 0] == b[3 * Z:3 * Z + 3, 3 * Y:3 * Y + 3, :].mean()


@pytest.mark.parametrize("i", range(19))
def test_coarse_pulled_moves_an_impulse_by_c_i(i):
    """A unit population i filling the fine box of coarse voxel X0 is pulled
    by the coarse voxel X0 + c_i (periodic) and by no other."""
    r, (nz, ny, nx) = 2, (4, 6, 8)                 # coarse box, axes (z, y, x)
    f = np.zeros((19, nz * r, ny * r, nx * r))
    X0 = (1, 2, 3)                                 # (z, y, x)
    f[i, X0[0] * r:(X0[0] + 1) * r, X0[1] * r:(X0[1] + 1) * r, X0[2] * r:(X0[2] + 1) * r] = 1.0
    out = cl.coarse_pulled(f, r)
    cxi, cyi, czi = (int(v) for v in L.C[i])
    want = np.zeros((19, nz, ny, nx))
    want[i, (X0[0] + czi) % nz, (X0[1] + cyi) % ny, (X0[2] + cxi) % nx] = 1.0
    assert np.array_equal(out, want)


def _shear_state(a, b, nu0, rho0=1.25, n=8, r=2, A=0.01, only=None):
    """Fine periodic equilibrium state whose box-filtered velocity is a shear
    u_b(X) = A sin(2 pi X_a / n) (X_a the coarse coordinate along axis a) and
    whose sub-filter stress is tau_ab = tau_ba = -2 rho0 nu0 S_ab, written
    in by a zero-mean fluctuation of u_a and u_b inside every r^3 box.
    Axes a, b: 0 = x, 1 = y, 2 = z.  Returns (f, D) with D(X) the central
    difference (u_b(X_a + 1) - u_b(X_a - 1)) / 2 on the coarse lattice, so
    S_ab = D / 2.  With `only` = (cov, X0): the fluctuation sits in the one
    box X0 = (z, y, x) with covariance cov, zero elsewhere."""
    N = n * r
    zyx = np.indices((n, n, n))                    # coarse (z, y, x)
    Xa = zyx[2 - a]
    ub = A * np.sin(2 * np.pi * Xa / n)
    D = 0.5 * (A * np.sin(2 * np.pi * (Xa + 1) / n) - A * np.sin(2 * np.pi * (Xa - 1) / n))
    cov = -nu0 * D                                 # <u'_a u'_b> = -2 nu0 S_ab
    if only is not None:
        c0, X0 = only
        cov = np.zeros((n, n, n))
        cov[X0] = c0
    up = lambda c: c.repeat(r, 0).repeat(r, 1).repeat(r, 2)
    # +1 / -1 on alternate fine x inside every box: zero box mean
    p = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)[None, None, :]
    al = np.sqrt(np.abs(cov))
    be = np.sign(cov) * al
    u = np.zeros((3, N, N, N))
    u[b] = up(ub) + up(be) * p
    u[a] = up(al) * p
    rho = np.full((N, N, N), rho0)
    return L.equilibrium(rho, u), D


@pytest.mark.parametrize("a,b", [(1, 0), (2, 0), (0, 1), (2, 1), (0, 2), (1, 2)])
@pytest.mark.parametrize("nu0", [0.01, -0.002])
def test_eddy_target_recovers_a_planted_eddy_viscosity(a, b, nu0):
    """Sub-filter stress exactly -2 rho nu0 S: the least-squares fit returns
    nu_t = nu0 in every neighbourhood, so d_tau = 3 nu0 (0.03 and -0.006,
    both inside the clamp for tau_c = 0.51).  A reversed central difference
    or a flipped -num/den gives -3 nu0; a dropped 3 gives nu0; a missing
    density in the denominator gives 1.25 x; a wrong axis gives 0."""
    f, _ = _shear_state(a, b, nu0)
    t = cl.eddy_target(f, 2, 0.51)
    assert np.allclose(t, 3 * nu0, rtol=1e-9, atol=1e-12), (t.min(), t.max())


def test_eddy_target_ignores_an_isotropic_sub_filter_stress():
    """The fit uses the deviator of the sub-filter stress.  Inside every 2^3
    box the fine velocity carries +-eps along each axis with the signs set by
    the subcell's x, y and z parity, so the eight subcells take all eight
    sign patterns: the sub-filter stress is rho eps^2 I (equal variances, no
    covariance).  Under the diverging filtered velocity u_x = A sin(2 pi X /
    n) (S_xx != 0) the target is 0 everywhere; keeping the trace would give
    3 nu_t = -3 sum_N rho eps^2 S_xx / (2 rho sum_N S_xx^2), about -5e-3."""
    n, r, A, eps, rho0 = 8, 2, 0.01, 0.004, 1.1
    N = n * r
    X = np.indices((n, n, n))[2]
    up = lambda c: c.repeat(r, 0).repeat(r, 1).repeat(r, 2)
    fine = np.indices((N, N, N))                   # fine (z, y, x)
    u = np.stack([eps * np.where(fine[2 - a] % 2 == 0, 1.0, -1.0) for a in range(3)])
    u[0] += up(A * np.sin(2 * np.pi * X / n))
    f = L.equilibrium(np.full((N, N, N), rho0), u)
    t = cl.eddy_target(f, r, 0.51)
    assert np.allclose(t, 0.0, rtol=0, atol=1e-12), (t.min(), t.max())


@pytest.mark.parametrize("nu0,want", [(0.3, 0.5), (-0.1, -(0.51 - 0.5) + 1e-3)])
def test_eddy_target_is_clamped(nu0, want):
    """A planted eddy viscosity whose 3 nu0 lies outside the admissible range
    gives the bound: at most 1/2, at least -(tau_c - 1/2) + 1e-3 (so that the
    coarse level keeps tau > 1/2)."""
    f, _ = _shear_state(0, 1, nu0)
    t = cl.eddy_target(f, 2, 0.51)
    assert np.allclose(t, want, rtol=0, atol=1e-15)


def test_eddy_target_sums_over_the_3x3x3_neighbourhood():
    """Sub-filter stress in one coarse voxel X0 only: the target is nonzero
    exactly on the 27 voxels whose neighbourhood holds X0, with the value
    -3 (2 tau_xy(X0) S_xy(X0)) / (4 rho sum_N S_xy^2), where the
    neighbourhood sum of S_xy^2 (S_xy depends on y only) is
    9 (S(y-1)^2 + S(y)^2 + S(y+1)^2)."""
    rho0, n, X0 = 1.25, 8, (3, 4, 5)
    _, D = _shear_state(1, 0, 0.0, rho0=rho0)
    S = D / 2                                      # S_xy as a field over (z, y, x)
    c0 = -0.06 * S[X0]                             # covariance in X0 (per unit density)
    f, _ = _shear_state(1, 0, 0.0, rho0=rho0, only=(c0, X0))
    t = cl.eddy_target(f, 2, 0.51)
    Sy = S[0, :, 0]                                # S_xy along y
    for z in range(n):
        for y in range(n):
            for x in range(n):
                near = all(min((p - q) % n, (q - p) % n) <= 1 for p, q in zip((z, y, x), X0))
                if near:
                    s2 = 9 * (Sy[(y - 1) % n] ** 2 + Sy[y] ** 2 + Sy[(y + 1) % n] ** 2)
                    want = -3 * (2 * rho0 * c0 * S[X0]) / (4 * rho0 * s2)
                else:
                    want = 0.0
                assert abs(t[z, y, x] - want) <= 1e-9 * abs(want) + 1e-14, ((z, y, x), t[z, y, x], want)


# ----------------------------------------------------------- training loop

def test_splitmix64_published_sequence():
    """The first outputs of the published SplitMix64 generator seeded with 0
    (its state advances by the golden-ratio increment per call)."""
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [cl.splitmix64((k * g) & ((1 << 64) - 1)) for k in range(3)]
    assert got == want


def test_minibatch_counter_layout():
    """Step k draws samples from counters seed + (k - 1) B .. seed + k B - 1."""
    idx = cl.minibatch_indices(5, 3, 4, 1000)
    assert list(idx) == [cl.splitmix64(5 + 8 + b) % 1000 for b in range(4)]
    assert np.all((idx >= 0) & (idx < 1000))


def test_train_one_step_is_adam_on_the_standardised_minibatch():
    """One step: the folded result equals Adam's first step (|update| = lr per
    parameter, sign of the minibatch gradient of the standardised problem),
    folded; a constant feature column keeps scale 1."""
    rng = np.random.default_rng(40)
    X = rng.standard_normal((300, 16)) * np.arange(1, 17) + 3.0
    X[:, 15] = 0.51                                        # constant (tau)
    t = 0.01 * X[:, 0] - 0.002 * X[:, 4] ** 2
    th0 = random_theta(41)
    got, _ = cl.train(X, t, th0, 1, 64, 1e-3, 9)
    mu, sd = X.mean(0), X.std(0)
    assert sd[15] < 1e-6 * 0.51          # rounding noise of a constant column
    sd[15] = 1.0
    idx = [cl.splitmix64(9 + b) % 300 for b in range(64)]
    _, g = cl.loss_and_grad(th0, (X[idx] - mu) / sd, (t[idx] - t.mean()) / t.std())
    step = th0 - 1e-3 * g / (np.abs(g) + 1e-8)
    want = cl.fold_normalisation(step, mu, sd, t.mean(), t.std())
    assert np.allclose(got, want, rtol=1e-12, atol=1e-15)


def test_train_steps_with_a_constant_gradient_move_by_lr_each():
    """Adam's bias-corrected moments of a constant gradient g are g and g^2
    at every step k (m_k = (1 - b1^k) g, v_k = (1 - b2^k) g^2), so each step
    moves a weight by lr g / (|g| + eps).  A one-sample training set makes
    every minibatch the same, and a learning rate of 1e-7 keeps the gradient
    constant over three steps; the weights then move by 3 lr g / (|g| + eps)
    (a step counter stuck at 1 would move them by 3.9 lr)."""
    rng = np.random.default_rng(44)
    X = rng.standard_normal((1, 16))
    t = np.array([0.7])
    th0 = random_theta(45)
    lr, K = 1e-7, 3
    got, _ = cl.train(X, t, th0, K, 8, lr, 3)
    # one sample: every column is constant (scale 1) and the standardised
    # problem has input 0 and target 0
    _, g = cl.loss_and_grad(th0, np.zeros((8, 16)), np.zeros(8))
    want = th0 - K * lr * g / (np.abs(g) + 1e-8)
    want = cl.fold_normalisation(want, X[0], np.ones(16), 0.7, 1.0)
    moved = np.abs(g) > 1e-4
    assert moved.sum() > 100
    assert np.allclose(got[moved], want[moved], rtol=0, atol=1e-4 * K * lr)


def test_train_lowers_the_loss():
    rng = np.random.default_rng(42)
    X = rng.standard_normal((2000, 16))
    t = np.tanh(X[:, 0] - 0.5 * X[:, 3])
    th0 = random_theta(43, scale=0.2)
    y0, _ = cl.forward(cl.fold_normalisation(th0, X.mean(0), X.std(0), t.mean(), t.std()), X)
    th, _ = cl.train(X, t, th0, 300, 128, 3e-3, 1)
    y1, _ = cl.forward(th, X)
    assert np.mean((y1 - t) ** 2) < 0.5 * np.mean((y0 - t) ** 2)
