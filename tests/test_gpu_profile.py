"""GPU: the per-kernel event profiler (tracing).

lbm_profile records a CUDA event pair around every kernel launch of a grid;
lbm_profile_read aggregates them per kernel and lbm_profile_trace returns
them one by one.  Both views must agree, count every launch of the steps
and the units (updated voxels) each launch covers, and the trace must keep
the steps in order."""
import numpy as np
import pytest

from cases import make_grid

from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_profile_stats_and_trace_agree(lbm):
    flags, bc = wl.cavity(0, dims=(64, 48, 40))
    g = make_grid(lbm, "dense", flags, bc, 0.6)
    lbm.lbm_init_equilibrium(g, 0, None, None)
    lbm.lbm_step(g, 2)
    lbm.lbm_profile(g, 1)
    lbm.lbm_step(g, 6)
    stats = lbm.lbm_profile_read(g)
    trace = lbm.lbm_profile_trace(g)
    lbm.lbm_profile(g, 0)
    n_upd = lbm.lbm_get_info(g)["n_updated"][0]
    n_lid = int(((flags & 7) == 2).sum())
    assert set(stats) == {"dense_interior", "dense_boundary"}
    assert stats["dense_interior"]["launches"] == stats["dense_boundary"]["launches"] == 6
    assert stats["dense_interior"]["units"] == 6 * (n_upd - n_lid)
    assert stats["dense_boundary"]["units"] == 6 * n_lid
    assert len(trace) == 12
    for name in stats:
        rec = [r for r in trace if r[0] == name]
        assert len(rec) == 6
        assert all(e >= s_ >= 0.0 for _, s_, e, _ in rec)
        total = sum(e - s_ for _, s_, e, _ in rec)
        assert abs(total - stats[name]["total_ms"]) <= 1e-3 + 1e-3 * total
    # steps run in order: each step's interior launch starts after the
    # previous one ended
    inter = [r for r in trace if r[0] == "dense_interior"]
    assert all(b[1] >= a[2] - 1e-3 for a, b in zip(inter, inter[1:]))
    lbm.lbm_grid_destroy(g)
