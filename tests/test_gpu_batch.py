"""GPU: the batched persistent step.

A batch must advance every case exactly as the case would advance on its own
(same arithmetic: populations bit-identical), match the FP64 oracle, survive
autotuning unchanged, and run the full 128-case serving workload.
"""
import numpy as np
import pytest

from cases import F32_RTOL, max_rel_err, run_oracle, updated_mask
from oracle import lbm as olbm
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def make_case(lbm, c, storage="f32"):
    nx, ny, nz = c["dims"]
    phys = lbm.physics(c["tau"], storage=storage, periodic=(1, 1, 1))
    if c["kind"] == "dense":
        g = lbm.lbm_grid_create_dense(c["dims"], phys)
        lbm.lbm_set_boundary(g, 0, c["flags"])
    else:
        g = lbm.lbm_grid_create_sparse(c["dims"], 8, c["flags"], phys)
    rho, u = wl.batch_case_fields(c)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    return g


SMALL = dict(n_cases=6, seed=31, lmin=16, lmax=48, max_solid=0.2)


def test_batch_equals_individual_runs(lbm):
    cases = wl.batch_cases(**SMALL)
    grids = [make_case(lbm, c) for c in cases]
    alone = [make_case(lbm, c) for c in cases]
    b = lbm.lbm_batch_create(grids)
    lbm.lbm_batch_step(b, 5)
    lbm.lbm_batch_step(b, 4)          # second graph, odd then even counts
    lbm.lbm_batch_step(b, 5)          # replay of the first graph
    for g in alone:
        lbm.lbm_step(g, 14)
    for c, g, a in zip(cases, grids, alone):
        m = updated_mask(c["flags"])
        fb = lbm.lbm_get_populations_f64(g, 0)
        fa = lbm.lbm_get_populations_f64(a, 0)
        assert np.array_equal(fb[:, m], fa[:, m]), c["kind"]
        assert lbm.lbm_get_info(g)["steps_done"] == 14


def test_batch_cases_match_oracle(lbm):
    cases = wl.batch_cases(n_cases=2, seed=32, lmin=16, lmax=32, max_solid=0.15)
    grids = [make_case(lbm, c) for c in cases]
    b = lbm.lbm_batch_create(grids)
    lbm.lbm_batch_step(b, 20)
    for c, g in zip(cases, grids):
        rho, u = wl.batch_case_fields(c)
        ref = run_oracle(c["flags"], None, rho, u, c["tau"], 20, periodic=(1, 1, 1))
        assert max_rel_err(lbm.lbm_get_populations_f64(g, 0), ref, c["flags"]) <= F32_RTOL


# FP16 storage rounds each stored population once per update; collision
# damps earlier roundings, so the relative velocity error stays near the
# format's unit roundoff: bound 4 u = 4 x 2^-11 (as for the other layouts)
F16_VEL_L2 = 4 * 2.0 ** -11


def fp16_cases():
    """Serving-batch cases at both ends of the tau range: dense and 8^3
    block-sparse, random spheres and boxes, a 64^3 case."""
    specs = [("dense", (64, 64, 64), 0.10, "spheres", 0.52),
             ("sparse", (48, 40, 56), 0.15, "boxes", 0.80),
             ("dense", (40, 32, 48), 0.20, "boxes", 0.66),
             ("sparse", (64, 48, 40), 0.05, "spheres", 0.52)]
    out = []
    for k, (kind, dims, frac, shape, tau) in enumerate(specs):
        nx, ny, nz = dims
        flags = wl.random_obstacles((nz, ny, nx), seed=170 + k, solid_fraction=frac, kind=shape)
        out.append({"kind": kind, "dims": dims, "flags": flags, "tau": tau, "u0": 0.02,
                    "solid_fraction": frac})
    return out


def test_fp16_batch_matches_oracle_and_individual_runs(lbm):
    """The FP16 serving form: 100 batched steps give every case the
    populations of the same case stepped alone bit for bit, and a velocity
    field within 4 unit roundoffs of FP16 (relative L2 over the fluid
    voxels) of the FP64 oracle."""
    cases = fp16_cases()
    grids = [make_case(lbm, c, "f16") for c in cases]
    alone = [make_case(lbm, c, "f16") for c in cases]
    b = lbm.lbm_batch_create(grids)
    lbm.lbm_batch_autotune(b, 2)
    lbm.lbm_batch_step(b, 100)
    for g in alone:
        lbm.lbm_step(g, 100)
    for c, g, a in zip(cases, grids, alone):
        m = updated_mask(c["flags"])
        fb = lbm.lbm_get_populations_f64(g, 0)
        assert np.array_equal(fb[:, m], lbm.lbm_get_populations_f64(a, 0)[:, m]), c["kind"]
        rho, u = wl.batch_case_fields(c)
        ref = run_oracle(c["flags"], None, rho, u, c["tau"], 100, periodic=(1, 1, 1))
        _, ur = olbm.state_moments(ref)
        _, ug = lbm.lbm_get_moments(g, 0)
        l2 = float(np.sqrt(((ug[:, m] - ur[:, m]) ** 2).sum() / (ur[:, m] ** 2).sum()))
        print(f"{c['kind']} {c['dims']} tau {c['tau']}: FP16 velocity L2 vs oracle {l2:.3e}")
        assert l2 <= F16_VEL_L2


def test_batch_autotune_restores_states(lbm):
    cases = wl.batch_cases(**SMALL)
    grids = [make_case(lbm, c) for c in cases]
    b = lbm.lbm_batch_create(grids)
    lbm.lbm_batch_step(b, 3)
    before = [lbm.lbm_get_populations_f64(g, 0) for g in grids]
    k, ms = lbm.lbm_batch_autotune(b, 4)
    assert k in (1, 2, 3, 4, 6, 8) and all(t > 0 for t in ms)
    for c, g, f0 in zip(cases, grids, before):
        m = updated_mask(c["flags"])
        assert np.array_equal(lbm.lbm_get_populations_f64(g, 0)[:, m], f0[:, m])
    assert lbm.lbm_batch_info(b)["ctas_per_sm"] == k


def test_batch_rejects_unsupported_cases(lbm):
    c = wl.batch_cases(n_cases=2, seed=33, lmin=16, lmax=16)
    g0 = make_case(lbm, c[0])
    g1 = make_case(lbm, c[1], storage="f16")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([g0, g1])
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    flags, bc = wl.cavity(0, dims=(16, 16, 16))
    gc = lbm.lbm_grid_create_dense((16, 16, 16), lbm.physics(0.6))
    lbm.lbm_set_boundary(gc, 0, flags, None, np.array([0.05, 0, 0, 1], np.float32))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([g0, gc])
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


def test_full_serving_batch_conserves_mass(lbm):
    """128 cases (32..160 per edge, half dense half sparse, up to 20 % solid,
    tau 0.52..0.8), FP16 storage: the batch runs and every case keeps its mass
    (periodic box with bounce-back obstacles)."""
    cases = wl.batch_cases()
    grids = [make_case(lbm, c, storage="f16") for c in cases]
    m0 = np.array([lbm.lbm_conservation(g)[0] for g in grids])
    b = lbm.lbm_batch_create(grids)
    info = lbm.lbm_batch_info(b)
    assert info["n_updated"] == sum(int(updated_mask(c["flags"]).sum()) for c in cases)
    lbm.lbm_batch_autotune(b, 4)
    lbm.lbm_batch_step(b, 10)
    m1 = np.array([lbm.lbm_conservation(g)[0] for g in grids])
    assert np.max(np.abs(m1 / m0 - 1)) <= 1e-5


def test_batch_closure_matches_oracle(lbm):
    """Closure on the cases whose largest edge is <= 24 (one dense, one
    sparse), the other two plain, in one batch; each case against the FP64
    oracle after 6 steps.  Closure cases: the oracle's closure step on the
    BF16-rounded network, tolerance the FP32 bar plus the oracle's response to
    a 2e-2 relative change of d_tau (the BF16 network's bound); plain cases:
    the FP32 bar."""
    from test_gpu_closure import he_init, storage_weights
    from oracle import closure as ocl
    from oracle import lbm as olbm
    cases = wl.batch_cases(n_cases=4, seed=38, lmin=16, lmax=32, max_solid=0.15)
    on = [max(c["dims"]) <= 24 for c in cases]
    assert on == [True, False, False, True]
    steps = 6
    grids, fields = [], []
    for k, c in enumerate(cases):
        nx, ny, nz = c["dims"]
        rho, u = wl.random_fields((nz, ny, nx), seed=130 + k, u_amp=0.02)
        phys = lbm.physics(c["tau"], periodic=(1, 1, 1))
        if c["kind"] == "dense":
            g = lbm.lbm_grid_create_dense(c["dims"], phys)
            lbm.lbm_set_boundary(g, 0, c["flags"])
        else:
            g = lbm.lbm_grid_create_sparse(c["dims"], 8, c["flags"], phys)
        lbm.lbm_init_equilibrium(g, 0, rho, u)
        grids.append(g)
        fields.append((rho, u))
    # network on the scale of this state's features, d_tau ~ 1e-2
    f0 = olbm.init_equilibrium(*fields[0], cases[0]["flags"])
    X = ocl.features(olbm.stream_with_walls(f0, cases[0]["flags"], (True,) * 3)[
        :, (cases[0]["flags"] & 7) == 0], cases[0]["tau"])
    sd = X.std(axis=0)
    sd[sd < 1e-9] = 1.0
    theta = he_init(131, scale_out=0.05)
    theta[:1024] = (theta[:1024].reshape(64, 16) / sd).ravel()
    theta = theta.astype(np.float32)
    th = storage_weights(theta)
    th_eps = th.copy()
    th_eps[5248:] *= 1 + 2e-2
    b = lbm.lbm_batch_create(grids)
    lbm.lbm_batch_closure_load(b, theta, 24)
    lbm.lbm_batch_step(b, steps)
    per = (True, True, True)
    for c, g, (rho, u), cl_on in zip(cases, grids, fields, on):
        f0 = olbm.init_equilibrium(rho, u, c["flags"])
        got = lbm.lbm_get_populations_f64(g, 0)
        if cl_on:
            ref = ocl.run(f0, c["flags"], c["tau"], th, steps, periodic=per)
            ref_eps = ocl.run(f0, c["flags"], c["tau"], th_eps, steps, periodic=per)
            plain = olbm.run(f0, c["flags"], c["tau"], steps, periodic=per)
            tol = F32_RTOL + max_rel_err(ref_eps, ref, c["flags"])
            effect = max_rel_err(plain, ref, c["flags"])
            err = max_rel_err(got, ref, c["flags"])
            print(f"{c['kind']} closure case: effect {effect:.3e}, GPU vs oracle {err:.3e}, "
                  f"tolerance {tol:.3e}")
            assert effect > 10 * tol
            assert err <= tol
        else:
            ref = olbm.run(f0, c["flags"], c["tau"], steps, periodic=per)
            assert max_rel_err(got, ref, c["flags"]) <= F32_RTOL
    # switching the closure off restores the plain kernel
    lbm.lbm_batch_closure_load(b, None, 0)
    assert lbm.lbm_batch_info(b)["n_items"] > 0
    lbm.lbm_batch_step(b, 1)
