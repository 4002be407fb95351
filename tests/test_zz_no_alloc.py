"""GPU: lbm_conservation_noalloc, the conservation sums for callers that cannot
allocate device memory.

Such callers (a solver loop that must never synchronise the device, which
cudaMalloc / cudaFree may do; an application whose device memory all belongs
to its own pool) pass the populations and a 4-double output that they own;
the entry point keeps its partial sums in a fixed device array inside the
library.  This file is collected last on purpose, so that a run stopping at
the first failure has run every other test first.  It checks the entry point,
called through the C ABI on a buffer the test owns, against the grid's own
lbm_conservation and against the FP64 oracle's sums of the same stored
populations (decoded here on the host), on two calls in a row (the second
call reuses the array the first one left behind), for both lattices and all
three storages, with and without flags; then its refusals: sizes beyond the
array, host pointers.
"""
import ctypes

import numpy as np
import pytest

from oracle import lattice as OL
from oracle import lbm as olbm
from paper_2503_07898_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# both sides are FP64 sums of the same values in different orders
REL_TOL = 1e-12


def _decode(raw, storage, q, shape):
    """Stored populations -> absolute FP64 f (q, nz, ny, nx): F32 is f itself,
    F16 / BF16 hold f_i - w_i."""
    if storage == "f32":
        f = raw.view(np.float32).astype(np.float64)
    elif storage == "f16":
        f = raw.view(np.float16).astype(np.float64)
    else:
        f = (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    f = f.reshape((q,) + shape)
    if storage != "f32":
        f = f + OL.lattice(q).W[:, None, None, None]
    return f


def _run_two_calls(lbm, g, storage, q, flags, with_flags):
    import torch
    nz, ny, nx = flags.shape
    n = nx * ny * nz
    nbytes = lbm.lbm_get_info(g)["population_bytes"][0]
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    flags_d = torch.from_numpy(np.ascontiguousarray(flags).ravel()).cuda() if with_flags else None
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        lbm.lbm_step(g, 7)
        ref = lbm.lbm_conservation(g)
        lbm.lbm_get_populations(g, 0, buf)
        out.fill_(float("nan"))
        lbm.lbm_conservation_noalloc(buf, storage, n, flags_d, out, stream, lattice=q)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        orc = olbm.conservation(_decode(buf.cpu().numpy(), storage, q, flags.shape),
                                flags if with_flags else None)
        for want in (ref, orc):
            assert abs(got[0] / want[0] - 1) <= REL_TOL, (call, got, want)
            assert np.all(np.abs(got[1:] - want[1:]) <= REL_TOL * want[0]), (call, got, want)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_noalloc_matches_conservation_on_two_calls(lbm, storage, q):
    """A walled cavity with an obstacle: flags select the updated voxels."""
    dims = (48, 40, 36)
    flags, bc = wl.cavity(0, dims=dims)
    flags[10:14, 8:12, 20:30] = wl.SOLID
    t = flags & 7
    g = lbm.lbm_grid_create_dense(dims, lbm.physics(0.6, storage=storage, lattice=q))
    lbm.lbm_set_boundary(g, 0, flags, np.ascontiguousarray(bc[:, t == 2].T, np.float32))
    rho, u = wl.random_fields(flags.shape, seed=90, u_amp=0.02)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    _run_two_calls(lbm, g, storage, q, flags, True)
    lbm.lbm_grid_destroy(g)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_noalloc_without_flags_on_a_periodic_box(lbm, storage):
    """flags = NULL sums every voxel (an all-fluid periodic grid)."""
    dims = (40, 24, 32)
    flags = np.zeros(dims[::-1], np.uint8)
    g = lbm.lbm_grid_create_dense(dims, lbm.physics(0.6, storage=storage, periodic=(1, 1, 1)))
    lbm.lbm_set_boundary(g, 0, flags)
    rho, u = wl.random_fields(flags.shape, seed=91, u_amp=0.02)
    lbm.lbm_init_equilibrium(g, 0, rho, u)
    _run_two_calls(lbm, g, storage, 19, flags, False)
    lbm.lbm_grid_destroy(g)


def test_noalloc_rejects_sizes_beyond_its_array(lbm):
    import torch
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    lib = lbm.load()
    st = lib.lbm_conservation_noalloc(ctypes.c_void_p(buf.data_ptr()), 0, 19,
                                      ctypes.c_int64(67_108_865), None,
                                      ctypes.c_void_p(out.data_ptr()), None)
    assert st == lbm.LBM_ERR_INVALID
    assert "67,108,864" in lbm.lbm_last_error()


def test_noalloc_rejects_host_pointers(lbm):
    """Host memory never reaches the kernels: the C entry point refuses it
    (cudaPointerGetAttributes) and the binding refuses CPU tensors."""
    import torch
    host = np.zeros(19 * 64, np.float32)
    out_d = torch.zeros(4, dtype=torch.float64, device="cuda")
    out_h = np.zeros(4, np.float64)
    buf_d = torch.zeros(19 * 64, dtype=torch.float32, device="cuda")
    lib = lbm.load()
    st = lib.lbm_conservation_noalloc(ctypes.c_void_p(host.ctypes.data), 0, 19, ctypes.c_int64(64),
                                      None, ctypes.c_void_p(out_d.data_ptr()), None)
    assert st == lbm.LBM_ERR_INVALID and "not device memory" in lbm.lbm_last_error()
    st = lib.lbm_conservation_noalloc(ctypes.c_void_p(buf_d.data_ptr()), 0, 19, ctypes.c_int64(64),
                                      None, ctypes.c_void_p(out_h.ctypes.data), None)
    assert st == lbm.LBM_ERR_INVALID and "not device memory" in lbm.lbm_last_error()
    with pytest.raises(ValueError):
        lbm.lbm_conservation_noalloc(torch.zeros(19 * 64), "f32", 64, None, out_d)
    with pytest.raises(ValueError):     # f shorter than 19 x n_voxels
        lbm.lbm_conservation_noalloc(buf_d, "f32", 65, None, out_d)
    with pytest.raises(ValueError):     # a 27-population buffer needs 27 x n_voxels
        lbm.lbm_conservation_noalloc(buf_d, "f32", 64, None, out_d, lattice=27)
