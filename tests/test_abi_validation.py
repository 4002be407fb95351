"""Argument checks of the C ABI (CPU, no GPU needed).

Every entry point validates its arguments on the host before it touches the
device, and reports a bad call as a status (never an abort) with a message
in lbm_last_error().  These calls all fail in that validation, so they run
without a GPU; the device paths behind them are exercised by the -m gpu
tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2503_07898_gb300 import binding as lbm


@pytest.fixture(scope="module")
def lib():
    from paper_2503_07898_gb300 import build
    build.build()
    return lbm.load()


def status_of(fn, *args):
    try:
        fn(*args)
    except lbm.LbmError as e:
        return e.status, str(e)
    return lbm.LBM_OK, ""


def dense(dims, phys):
    return lbm.lbm_grid_create_dense(dims, phys, allocator=False, stream=0)


@pytest.mark.parametrize("kw,status,text", [
    (dict(tau=0.5), lbm.LBM_ERR_INVALID, "tau must be > 0.5"),
    (dict(tau=0.49), lbm.LBM_ERR_INVALID, "tau must be > 0.5"),
    (dict(tau=float("nan")), lbm.LBM_ERR_INVALID, "tau must be > 0.5"),
    (dict(tau=float("inf")), lbm.LBM_ERR_INVALID, "tau must be > 0.5"),
    (dict(tau=0.6, collision=2), lbm.LBM_ERR_INVALID, "unknown collision"),
    (dict(tau=0.6, storage=3), lbm.LBM_ERR_INVALID, "unknown storage"),
    (dict(tau=0.6, schedule=3), lbm.LBM_ERR_INVALID, "unknown schedule"),
    (dict(tau=0.6, lattice=15), lbm.LBM_ERR_INVALID, "lattice must be 19 or 27"),
    (dict(tau=0.6, closure=1), lbm.LBM_ERR_UNSUPPORTED, "multi-resolution"),
    (dict(tau=0.6, schedule="bitmask"), lbm.LBM_ERR_UNSUPPORTED, "block-sparse"),
])
def test_dense_creation_rejects_bad_physics(lib, kw, status, text):
    st, msg = status_of(dense, (8, 8, 8), lbm.physics(**kw))
    assert st == status, msg
    assert text in msg and text in lbm.lbm_last_error()


@pytest.mark.parametrize("dims", [(0, 8, 8), (8, -1, 8), (8, 8, 0)])
def test_dense_creation_rejects_bad_dims(lib, dims):
    st, msg = status_of(dense, dims, lbm.physics(0.6))
    assert st == lbm.LBM_ERR_INVALID and "dims must be positive" in msg


def test_null_pointers_are_refused(lib):
    out = C.c_void_p()
    dims = (C.c_int * 3)(8, 8, 8)
    phys = lbm.physics(0.6)
    assert lib.lbm_grid_create_dense(None, C.byref(phys), None, None, C.byref(out)) == \
        lbm.LBM_ERR_INVALID
    assert lib.lbm_grid_create_dense(dims, None, None, None, C.byref(out)) == lbm.LBM_ERR_INVALID
    assert "physics is NULL" in lbm.lbm_last_error()
    assert lib.lbm_grid_create_dense(dims, C.byref(phys), None, None, None) == lbm.LBM_ERR_INVALID
    assert "out is NULL" in lbm.lbm_last_error()
    assert out.value is None
    # an allocator must give both callbacks
    half = lbm.lbm_allocator(None, lbm._ALLOC(), lbm._FREE())
    assert lib.lbm_grid_create_dense(dims, C.byref(phys), C.byref(half), None, C.byref(out)) == \
        lbm.LBM_ERR_INVALID
    assert "allocator needs alloc and free" in lbm.lbm_last_error()


def test_calls_on_a_null_grid_are_refused(lib):
    info = lbm.lbm_info()
    d = C.c_double * 4
    for call in (lambda: lib.lbm_grid_destroy(None),
                 lambda: lib.lbm_get_info(None, C.byref(info)),
                 lambda: lib.lbm_set_schedule(None, 0),
                 lambda: lib.lbm_set_variant(None, 1),
                 lambda: lib.lbm_set_wait_limit(None, 0),
                 lambda: lib.lbm_set_boundary(None, 0, None, None, None),
                 lambda: lib.lbm_init_equilibrium(None, 0, None, None, 0),
                 lambda: lib.lbm_step(None, 1, None),
                 lambda: lib.lbm_sync(None),
                 lambda: lib.lbm_get_moments(None, 0, None, None, 0),
                 lambda: lib.lbm_conservation(None, d()),
                 lambda: lib.lbm_profile(None, 1),
                 lambda: lib.lbm_closure_load(None, None, 0),
                 lambda: lib.lbm_batch_destroy(None),
                 lambda: lib.lbm_batch_step(None, 1, None)):
        assert call() == lbm.LBM_ERR_INVALID
        assert lbm.lbm_last_error() != ""


def test_batch_creation_needs_cases(lib):
    out = C.c_void_p()
    assert lib.lbm_batch_create(0, None, C.byref(out)) == lbm.LBM_ERR_INVALID
    assert "bad batch arguments" in lbm.lbm_last_error()


def test_sparse_creation_checks(lib):
    flags = np.zeros((8, 8, 12), np.uint8)
    mk = lambda edge, fl, phys: lbm.lbm_grid_create_sparse((12, 8, 8), edge, fl, phys,
                                                           allocator=False, stream=0)
    st, msg = status_of(mk, 6, flags, lbm.physics(0.6))
    assert st == lbm.LBM_ERR_INVALID and "block_edge must be 4 or 8" in msg
    st, msg = status_of(mk, 8, flags, lbm.physics(0.6, periodic=(1, 0, 0)))
    assert st == lbm.LBM_ERR_INVALID and "periodic axes need dims divisible" in msg
    st, msg = status_of(mk, 8, flags, lbm.physics(0.6, closure=1))
    assert st == lbm.LBM_ERR_UNSUPPORTED
    out = C.c_void_p()
    phys = lbm.physics(0.6)
    assert lib.lbm_grid_create_sparse((C.c_int * 3)(12, 8, 8), 8, None, C.byref(phys), None,
                                      None, C.byref(out)) == lbm.LBM_ERR_INVALID
    assert "sparse grids need flags" in lbm.lbm_last_error()


@pytest.mark.parametrize("dims,n_levels,lmap,status,text", [
    ((32, 32, 32), 0, np.zeros((1, 1, 1)), lbm.LBM_ERR_INVALID, "n_levels must be 1..4"),
    ((32, 32, 32), 5, np.zeros((1, 1, 1)), lbm.LBM_ERR_INVALID, "n_levels must be 1..4"),
    ((32, 32, 40), 3, np.zeros((1, 1, 1)), lbm.LBM_ERR_INVALID, "multiples of 8*2^(n_levels-1)"),
    ((32, 32, 96), 3, np.array([3, 2, 2]).reshape(3, 1, 1), lbm.LBM_ERR_INVALID,
     "level map value >= n_levels"),
    ((32, 32, 96), 3, np.array([0, 2, 2]).reshape(3, 1, 1), lbm.LBM_ERR_INVALID,
     "2:1 grading"),
])
def test_multires_creation_checks(lib, dims, n_levels, lmap, status, text):
    st, msg = status_of(lbm.lbm_grid_create_multires, dims, n_levels, lmap,
                        lbm.physics(0.6, periodic=(1, 1, 1)), False, 0)
    assert st == status and text in msg, msg


def test_multires_walls_only_next_to_the_finest_level(lib):
    """A walled side (z not periodic) must be owned by level 0."""
    lmap = np.array([1, 0, 0, 1], np.uint8).reshape(4, 1, 1)
    st, msg = status_of(lbm.lbm_grid_create_multires, (16, 16, 64), 2, lmap,
                        lbm.physics(0.6, periodic=(1, 1, 0)), False, 0)
    assert st == lbm.LBM_ERR_UNSUPPORTED and "non-periodic side must be level 0" in msg


@pytest.mark.parametrize("args,text", [
    (dict(storage=3), "unknown storage"),
    (dict(lattice=21), "lattice must be 19 or 27"),
    (dict(n=0), "n_voxels must be positive"),
    (dict(n=(1 << 26) + 1), "no-allocation limit of 67,108,864 voxels"),
])
def test_noalloc_sums_check_sizes_before_any_device_call(lib, args, text):
    kw = dict(storage=0, lattice=19, n=64)
    kw.update(args)
    out = (C.c_double * 4)()
    buf = C.c_void_p(16)   # never dereferenced: every call here fails its checks first
    assert lib.lbm_conservation_noalloc(buf, kw["storage"], kw["lattice"], C.c_int64(kw["n"]),
                                        None, out, None) == lbm.LBM_ERR_INVALID
    assert text in lbm.lbm_last_error()


def test_closure_entry_points_check_arguments(lib):
    assert lib.lbm_closure_forward(None, None, C.c_int64(0), 0, None, None) == lbm.LBM_ERR_INVALID
    assert lib.lbm_closure_train(None, None, C.c_int64(0), 0, 0, C.c_float(0), C.c_uint64(0),
                                 None, None, None) == lbm.LBM_ERR_INVALID
    assert lib.lbm_closure_dataset(None, 2, C.c_double(0.51), None, None) == lbm.LBM_ERR_INVALID


def test_each_call_replaces_the_last_error(lib):
    assert lib.lbm_step(None, 1, None) == lbm.LBM_ERR_INVALID
    assert lbm.lbm_last_error() != ""
    # creation starts by clearing the message, then fails on the new call's own check
    st, _ = status_of(dense, (0, 1, 1), lbm.physics(0.6))
    assert st == lbm.LBM_ERR_INVALID and lbm.lbm_last_error() == "dims must be positive"
