"""GPU: lbm_conservation_noalloc, the conservation sums for callers that cannot
allocate device memory.

Such callers (a solver loop that must never synchronise the device, which
cudaMalloc / cudaFree may do; an application whose device memory all belongs
to its own pool) pass the populations and a 4-double output that they own;
the entry point keeps its partial sums in a fixed device array inside the
library.  This file is collected last on purpose, so that a run stopping at
the first failure has run every other test first.  It checks the entry point,
called through the C ABI on a buffer the test owns, against the grid's own
lbm_conservation on two calls in a row (the second call reuses the array the
first one left behind), and its size limit.
"""
import numpy as np
import pytest

from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# both sides are FP64 sums of the same values in different orders
REL_TOL = 1e-12


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_noalloc_matches_conservation_on_two_calls(lbm, storage):
    import torch
    dims = (48, 40, 36)
    flags, bc = wl.cavity(0, dims=dims)
    flags[10:14, 8:12, 20:30] = wl.SOLID
    t = flags & 7
    g = lbm.lbm_grid_create_dense(dims, lbm.physics(0.6, storage=storage))
    lbm.lbm_set_boundary(g, 0, flags, np.ascontiguousarray(bc[:, t == 2].T, np.float32))
    rho, u = wl.random_fields(flags.shape, seed=90)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    n = dims[0] * dims[1] * dims[2]
    nbytes = lbm.lbm_get_info(g)["population_bytes"][0]
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    flags_d = torch.from_numpy(np.ascontiguousarray(flags).ravel()).cuda()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        lbm.lbm_step(g, 7)
        ref = lbm.lbm_conservation(g)
        lbm.lbm_get_populations(g, 0, buf)
        out.fill_(float("nan"))
        lbm.lbm_conservation_noalloc(buf, storage, n, flags_d, out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] / ref[0] - 1) <= REL_TOL, (call, got, ref)
        assert np.all(np.abs(got[1:] - ref[1:]) <= REL_TOL * ref[0]), (call, got, ref)


def test_noalloc_rejects_sizes_beyond_its_array(lbm):
    import torch
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_conservation_noalloc(buf, "f32", 67_108_865, None, out)
    assert e.value.status == lbm.LBM_ERR_INVALID
    assert "67,108,864" in str(e.value)
