"""GPU: interior-kernel variants, the autotuner, and FP16 / BF16 shifted storage.

Variants (16-byte vectors, scalar, 8-byte vectors, 4-byte vectors) must give the same
populations and match the oracle.  Shifted 16-bit storage (s = f - w, RN-even)
is compared with the FP64 oracle by the velocity-field L2 error; the bounds
follow from the storage rounding: one FP16 rounding of |s| <~ 5e-3 costs
~2.4e-6 per population and step, ~7e-5 in u after 100 steps of random-walk
accumulation, i.e. ~4e-3 relative to |u| ~ 0.02 (BF16: 8x coarser).
"""
import numpy as np
import pytest

from cases import F32_RTOL, make_grid, max_rel_err, run_oracle, updated_mask, velocity_l2
from oracle import lbm as olbm
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

F16_VEL_L2 = 1e-2
BF16_VEL_L2 = 6e-2


def run_variant(lbm, flags, bc, rho, u, tau, steps, variant, storage="f32", periodic=(0, 0, 0),
                collision="bgk"):
    g = make_grid(lbm, "dense", flags, bc, tau, collision, storage, periodic)
    lbm.lbm_set_variant(g, variant)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, steps)
    return g, lbm.lbm_get_populations_f64(g, 0)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_variants_identical_cavity(lbm, storage):
    flags, bc = wl.cavity(0, dims=(64, 24, 20))
    rho, u = wl.random_fields(flags.shape, seed=40, u_amp=0.02)
    outs = [run_variant(lbm, flags, bc, rho, u, 0.55, 50, v, storage)[1] for v in (0, 1, 2, 3)]
    m = updated_mask(flags)
    for o in outs[1:]:
        assert np.max(np.abs(o[:, m] - outs[0][:, m])) <= 1e-6


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("collision", ["bgk", "reg"])
def test_vector_kernel_parity(lbm, variant, collision):
    """Every dense interior variant (16-, 8-, 4-byte vectors and the scalar
    kernel the autotuner may pick) against the oracle after 100 steps:
    x-periodic wrap through the shuffles (periodic box) and x walls (cavity)."""
    dims_zyx = (12, 20, 64)
    rho, u = wl.random_fields(dims_zyx, seed=41)
    flags = np.zeros(dims_zyx, np.uint8)
    _, f = run_variant(lbm, flags, None, rho, u, 0.6, 100, variant, periodic=(1, 1, 1),
                       collision=collision)
    ref = run_oracle(flags, None, rho, u, 0.6, 100, collision, periodic=(1, 1, 1))
    assert max_rel_err(f, ref, flags) <= F32_RTOL
    flags, bc = wl.cavity(0, dims=(96, 20, 14))
    rho, u = wl.random_fields(flags.shape, seed=42, u_amp=0.02)
    _, f = run_variant(lbm, flags, bc, rho, u, 0.58, 100, variant, collision=collision)
    ref = run_oracle(flags, bc, rho, u, 0.58, 100, collision)
    assert max_rel_err(f, ref, flags) <= F32_RTOL


def test_vector_kernel_partial_warp(lbm):
    """x extent that is a multiple of the vector length but not of a warp's span."""
    flags, bc = wl.cavity(0, dims=(40, 9, 7))
    rho, u = wl.random_fields(flags.shape, seed=43, u_amp=0.02)
    _, f = run_variant(lbm, flags, bc, rho, u, 0.6, 100, 0)
    ref = run_oracle(flags, bc, rho, u, 0.6, 100)
    assert max_rel_err(f, ref, flags) <= F32_RTOL


@pytest.mark.parametrize("storage,bound", [("f16", F16_VEL_L2), ("bf16", BF16_VEL_L2)])
def test_shifted_storage_velocity_error(lbm, storage, bound):
    n, tau = 32, 0.6
    rho, u = wl.taylor_green_2d(n)
    flags = np.zeros((n, n, n), np.uint8)
    g, _ = run_variant(lbm, flags, None, rho, u, tau, 100, 0, storage, periodic=(1, 1, 1))
    _, v = lbm.lbm_get_moments(g, 0)
    ref = run_oracle(flags, None, rho, u, tau, 100, periodic=(1, 1, 1))
    _, vr = olbm.state_moments(ref)
    err = velocity_l2(v, vr, flags)
    print(f"{storage} Taylor-Green velocity L2 error after 100 steps: {err:.3e}")
    assert err <= bound
    flags, bc = wl.cavity(0, dims=(48, 24, 20))
    rho, u = wl.random_fields(flags.shape, seed=44, u_amp=0.02)
    g, _ = run_variant(lbm, flags, bc, rho, u, 0.58, 100, 0, storage)
    _, v = lbm.lbm_get_moments(g, 0)
    _, vr = olbm.state_moments(run_oracle(flags, bc, rho, u, 0.58, 100))
    err = velocity_l2(v, vr, flags)
    print(f"{storage} cavity velocity L2 error after 100 steps: {err:.3e}")
    assert err <= bound


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_shifted_storage_mass_drift(lbm, storage):
    dims_zyx = (16, 16, 32)
    rho, u = wl.random_fields(dims_zyx, seed=45)
    flags = np.zeros(dims_zyx, np.uint8)
    g = make_grid(lbm, "dense", flags, None, 0.6, storage=storage, periodic=(1, 1, 1))
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    m0 = lbm.lbm_conservation(g)
    lbm.lbm_step(g, 100)
    m1 = lbm.lbm_conservation(g)
    drift = abs(m1[0] - m0[0]) / m0[0]
    print(f"{storage} relative mass drift over 100 steps: {drift:.3e}")
    assert drift <= (1e-5 if storage == "f16" else 1e-4)


def test_autotune_restores_state(lbm):
    flags, bc = wl.cavity(0, dims=(64, 32, 24))
    rho, u = wl.random_fields(flags.shape, seed=46, u_amp=0.02)
    g = make_grid(lbm, "dense", flags, bc, 0.6)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_step(g, 5)
    before = lbm.lbm_get_populations_f64(g, 0)
    chosen, ms = lbm.lbm_autotune(g, 10)
    assert chosen in (0, 1, 2, 3) and all(t > 0 for t in ms[:4]) and ms[4] == 0
    after = lbm.lbm_get_populations_f64(g, 0)
    m = updated_mask(flags)
    assert np.array_equal(before[:, m], after[:, m])
    assert lbm.lbm_get_info(g)["steps_done"] == 5


def test_autotune_on_multires_restores_state(lbm):
    """On an 8^3-block multi-resolution grid the autotuner times the default
    lean kernel and its staged form, restores every level's state and keeps
    the faster one."""
    lmap = np.array([2, 1, 0, 1], np.uint8).reshape(4, 1, 1)
    dims = (32, 32, 128)
    g = lbm.lbm_grid_create_multires(dims, 3, lmap, lbm.physics(0.6, periodic=(1, 1, 1)))
    for lv in range(3):
        nx, ny, nz = (d >> lv for d in dims)
        rho, u = wl.random_fields((nz, ny, nx), seed=47 + lv, u_amp=0.02)
        lbm.lbm_init_equilibrium(g, lv, rho, u)
    lbm.lbm_step(g, 2)
    before = [lbm.lbm_get_populations_f64(g, lv) for lv in range(3)]
    chosen, ms = lbm.lbm_autotune(g, 4)
    assert chosen in (lbm.LBM_VARIANT_SCALAR, lbm.LBM_VARIANT_STAGED)
    assert ms[lbm.LBM_VARIANT_SCALAR] > 0 and ms[lbm.LBM_VARIANT_STAGED] > 0
    assert ms[0] == ms[2] == ms[3] == 0
    for lv in range(3):
        assert np.array_equal(lbm.lbm_get_populations_f64(g, lv), before[lv], equal_nan=True)
