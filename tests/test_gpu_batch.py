"""GPU: the batched persistent step.

A batch must advance every case exactly as the case would advance on its own
(same arithmetic: populations bit-identical), match the FP64 oracle, survive
autotuning unchanged, and run the full 128-case serving workload.
"""
import numpy as np
import pytest

from cases import F32_RTOL, max_rel_err, run_oracle, updated_mask
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
