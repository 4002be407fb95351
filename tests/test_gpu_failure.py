"""GPU: failure detection without a GPU fault.

The staged block-sparse kernel waits (on an mbarrier) for the bulk copy of
its block; the wait is bounded by time.  Here the limit is set to zero, so
every CTA's wait runs out at once while its copy is still in flight: the
step must latch LBM_ERR_TIMEOUT, lbm_sync must report it once and clear it,
and each CTA must have drained its copy before leaving (the context stays
usable and the next steps, with the default limit restored, equal the
default kernel's bit for bit).
"""
import numpy as np
import pytest

from cases import make_grid, updated_mask
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _channel():
    return wl.sphere_channel(dims=(76, 44, 44), radius_channel=19, sphere_center_x=22,
                             sphere_radius=8, u_in=0.04)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_staged_wait_timeout_is_latched_and_recovers(lbm, storage):
    flags, bc = _channel()
    rho, u = wl.random_fields(flags.shape, seed=160, u_amp=0.02)
    g = make_grid(lbm, "sparse", flags, bc, 0.56, storage=storage)
    lbm.lbm_set_variant(g, lbm.LBM_VARIANT_STAGED)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    lbm.lbm_sync(g)
    lbm.lbm_set_wait_limit(g, 0)
    lbm.lbm_step(g, 3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_sync(g)
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    lbm.lbm_sync(g)                       # reported once, then cleared
    # default limit again: the same grid, re-initialised, steps like the
    # default kernel
    lbm.lbm_set_wait_limit(g, -1)
    ref = make_grid(lbm, "sparse", flags, bc, 0.56, storage=storage)
    out = []
    for h in (g, ref):
        lbm.lbm_init_equilibrium(h, 0, rho, u)
        lbm.lbm_step(h, 20)
        lbm.lbm_sync(h)
        out.append(lbm.lbm_get_populations_f64(h, 0))
    m = updated_mask(flags)
    assert np.array_equal(out[0][:, m], out[1][:, m])
    lbm.lbm_grid_destroy(g)
    lbm.lbm_grid_destroy(ref)


def test_wait_limit_needs_a_grid(lbm):
    import ctypes
    assert lbm.load().lbm_set_wait_limit(None, ctypes.c_int64(0)) == lbm.LBM_ERR_INVALID
