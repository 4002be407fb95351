"""ctypes binding of liblbm (include/lbm.h), same function names as the C ABI.

Argument marshalling only: every step of the lattice-Boltzmann path runs in
the library's CUDA kernels.  PyTorch provides device memory (through the
``lbm_allocator`` hook, backed by its caching allocator) and streams.
Arrays may be numpy (host, ``device_ptrs = 0``) or CUDA torch tensors
(device, ``device_ptrs = 1``).  There is no CPU fallback: if ``liblbm.so`` is
missing, ``load()`` raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_ERR_INVALID, LBM_ERR_OOM, LBM_ERR_CUDA = 0, 1, 2, 3
LBM_ERR_TIMEOUT, LBM_ERR_DIVERGED, LBM_ERR_UNSUPPORTED, LBM_ERR_INTERNAL = 4, 5, 6, 7
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_INVALID", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA",
                4: "LBM_ERR_TIMEOUT", 5: "LBM_ERR_DIVERGED", 6: "LBM_ERR_UNSUPPORTED",
                7: "LBM_ERR_INTERNAL"}
LBM_COLLISION_BGK, LBM_COLLISION_REG = 0, 1
LBM_STORAGE_F32, LBM_STORAGE_F16, LBM_STORAGE_BF16 = 0, 1, 2
LBM_SCHEDULE_DISAGGREGATED, LBM_SCHEDULE_MONOLITHIC = 0, 1
LBM_LAYOUT_FLAGS, LBM_LAYOUT_BLOCK_COORDS, LBM_LAYOUT_NBR = 0, 1, 2
LBM_LAYOUT_BLOCK_MAP, LBM_LAYOUT_XNBR_COARSE, LBM_LAYOUT_XNBR_FINE = 3, 4, 5
LBM_LAYOUT_BOUNDARY_BITS, LBM_LAYOUT_BC_INDEX = 6, 7
LBM_LAYOUT_IFACE_SLOTS, LBM_LAYOUT_IFACE_CROSS = 8, 9
SCHEDULES = {"disaggregated": 0, "monolithic": 1, "bitmask": 2}


class lbm_physics(C.Structure):
    _fields_ = [("tau", C.c_double), ("collision", C.c_int), ("storage", C.c_int),
                ("closure", C.c_int), ("periodic", C.c_int * 3), ("schedule", C.c_int),
                ("lattice", C.c_int)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class lbm_allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", _ALLOC), ("free", _FREE)]


class lbm_info(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_levels", C.c_int), ("dims", C.c_int * 3),
                ("block_edge", C.c_int), ("n_updated", C.c_int64 * 4),
                ("n_blocks", C.c_int64 * 4), ("n_group_b", C.c_int64 * 4),
                ("n_regularized", C.c_int64), ("population_bytes", C.c_size_t * 4),
                ("steps_done", C.c_int64), ("lattice", C.c_int)]


class lbm_kernel_trace(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("start_ms", C.c_double), ("end_ms", C.c_double),
                ("units", C.c_int64)]


class lbm_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("units", C.c_int64)]


class LbmError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load liblbm.so (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2503_07898_gb300.build.build() "
                           "(nvcc, sm_103a). There is no CPU fallback.")
    lib = C.CDLL(LIB_PATH)
    P, I, vp = C.POINTER, C.c_int, C.c_void_p
    sig = {
        "lbm_grid_create_dense": [P(I), P(lbm_physics), P(lbm_allocator), vp, P(vp)],
        "lbm_grid_create_sparse": [P(I), I, vp, P(lbm_physics), P(lbm_allocator), vp, P(vp)],
        "lbm_grid_create_multires": [P(I), I, vp, P(lbm_physics), P(lbm_allocator), vp, P(vp)],
        "lbm_grid_destroy": [vp],
        "lbm_get_info": [vp, P(lbm_info)],
        "lbm_set_schedule": [vp, I],
        "lbm_set_boundary": [vp, I, vp, vp, vp],
        "lbm_init_equilibrium": [vp, I, vp, vp, I],
        "lbm_step": [vp, I, vp],
        "lbm_get_moments": [vp, I, vp, vp, I],
        "lbm_get_populations": [vp, I, vp, C.c_size_t, I],
        "lbm_set_populations": [vp, I, vp, C.c_size_t, I],
        "lbm_get_populations_f64": [vp, I, vp, I],
        "lbm_layout_bytes": [vp, I, I, P(C.c_size_t)],
        "lbm_get_layout": [vp, I, I, vp, C.c_size_t],
        "lbm_conservation": [vp, P(C.c_double)],
        "lbm_sync": [vp],
        "lbm_set_variant": [vp, I],
        "lbm_set_wait_limit": [vp, C.c_int64],
        "lbm_autotune": [vp, I, P(I), P(C.c_double)],
        "lbm_conservation_noalloc": [vp, I, I, C.c_int64, vp, vp, vp],
        "lbm_closure_dataset": [vp, I, C.c_double, vp, vp],
        "lbm_closure_train": [vp, vp, C.c_int64, I, I, C.c_float, C.c_uint64, vp, vp, vp],
        "lbm_closure_grad": [vp, vp, vp, vp, I, vp, vp, vp],
        "lbm_closure_forward": [vp, vp, C.c_int64, I, vp, vp],
        "lbm_closure_load": [vp, vp, C.c_size_t],
        "lbm_batch_create": [I, vp, P(vp)],
        "lbm_batch_destroy": [vp],
        "lbm_batch_step": [vp, I, vp],
        "lbm_batch_autotune": [vp, I, P(I), P(C.c_double)],
        "lbm_batch_info": [vp, P(C.c_int64), P(C.c_int64), P(I)],
        "lbm_batch_closure_load": [vp, vp, C.c_size_t, I],
        "lbm_profile": [vp, I],
        "lbm_profile_read": [vp, P(lbm_kernel_stat), I, P(I)],
        "lbm_profile_trace": [vp, P(lbm_kernel_trace), I, P(I)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.lbm_last_error.argtypes = []
    lib.lbm_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def lbm_last_error():
    return load().lbm_last_error().decode()


def _check(status, where):
    if status != LBM_OK:
        raise LbmError(status, where, lbm_last_error())


# ------------------------------------------------------------------- memory

class TorchAllocator:
    """lbm_allocator backed by the PyTorch CUDA caching allocator."""

    def __init__(self, device=None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.live = {}
        self._alloc_cb = _ALLOC(self._alloc)
        self._free_cb = _FREE(self._free)
        self.struct = lbm_allocator(None, self._alloc_cb, self._free_cb)

    def _alloc(self, ctx, nbytes, stream):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ctx, p, stream):
        self.live.pop(p, None)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(a, dtype):
    """(pointer, device_ptrs, keepalive) of a numpy array or CUDA tensor."""
    if a is None:
        return None, 0, None
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        if not a.is_contiguous():
            raise ValueError("device tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), 1, a
    if hasattr(a, "data_ptr"):  # CPU tensor (possibly pinned)
        if not a.is_contiguous():
            raise ValueError("host tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), 0, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), 0, arr


def physics(tau, collision="bgk", storage="f32", periodic=(0, 0, 0), schedule="disaggregated",
            closure=0, lattice=19):
    p = lbm_physics()
    p.tau = float(tau)
    p.collision = {"bgk": 0, "reg": 1}[collision] if isinstance(collision, str) else int(collision)
    p.storage = ({"f32": 0, "f16": 1, "bf16": 2}[storage] if isinstance(storage, str)
                 else int(storage))
    p.closure = int(closure)
    for a in range(3):
        p.periodic[a] = int(bool(periodic[a]))
    p.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    p.lattice = int(lattice)
    return p


class Grid:
    """Handle returned by lbm_grid_create_*; keeps the allocator alive."""

    def __init__(self, ptr, allocator, dims):
        self.ptr = ptr
        self.allocator = allocator
        self.dims = tuple(dims)

    @property
    def _as_parameter_(self):
        return self.ptr

    def __del__(self):
        try:
            if getattr(self, "ptr", None) and _lib is not None:
                _lib.lbm_grid_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass


def _alloc_arg(allocator):
    """TorchAllocator by default; False selects the library's cudaMalloc."""
    if allocator is None:
        allocator = TorchAllocator()
    return allocator, (None if allocator is False else C.byref(allocator.struct))


def lbm_grid_create_dense(dims, phys, allocator=None, stream=None):
    lib = load()
    alloc, ap = _alloc_arg(allocator)
    out = C.c_void_p()
    _check(lib.lbm_grid_create_dense((C.c_int * 3)(*dims), C.byref(phys), ap, _stream_ptr(stream),
                                     C.byref(out)), "lbm_grid_create_dense")
    return Grid(out, alloc, dims)


def lbm_grid_create_sparse(dims, block_edge, flags, phys, allocator=None, stream=None):
    lib = load()
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    if fl.size != dims[0] * dims[1] * dims[2]:
        raise ValueError("flags must cover the virtual box")
    alloc, ap = _alloc_arg(allocator)
    out = C.c_void_p()
    _check(lib.lbm_grid_create_sparse((C.c_int * 3)(*dims), int(block_edge),
                                      C.c_void_p(fl.ctypes.data), C.byref(phys), ap,
                                      _stream_ptr(stream), C.byref(out)), "lbm_grid_create_sparse")
    return Grid(out, alloc, dims)


def lbm_grid_create_multires(finest_dims, n_levels, level_map, phys, allocator=None, stream=None):
    """level_map: (mz, my, mx) array of owning levels per cube of 8*2^(n_levels-1)
    finest voxels."""
    lib = load()
    lm = np.ascontiguousarray(level_map, dtype=np.uint8)
    alloc, ap = _alloc_arg(allocator)
    out = C.c_void_p()
    _check(lib.lbm_grid_create_multires((C.c_int * 3)(*finest_dims), int(n_levels),
                                        C.c_void_p(lm.ctypes.data), C.byref(phys), ap,
                                        _stream_ptr(stream), C.byref(out)),
           "lbm_grid_create_multires")
    return Grid(out, alloc, finest_dims)


def lbm_grid_destroy(grid):
    if grid.ptr:
        _check(load().lbm_grid_destroy(grid.ptr), "lbm_grid_destroy")
        grid.ptr = None


def lbm_get_info(grid):
    info = lbm_info()
    _check(load().lbm_get_info(grid.ptr, C.byref(info)), "lbm_get_info")
    L = info.n_levels
    return {"kind": info.kind, "n_levels": L, "dims": tuple(info.dims),
            "block_edge": info.block_edge, "n_updated": list(info.n_updated)[:L],
            "n_blocks": list(info.n_blocks)[:L], "n_group_b": list(info.n_group_b)[:L],
            "n_regularized": info.n_regularized,
            "population_bytes": list(info.population_bytes)[:L], "steps_done": info.steps_done,
            "lattice": info.lattice}


def lbm_set_schedule(grid, schedule):
    s = SCHEDULES[schedule] if isinstance(schedule, str) else schedule
    _check(load().lbm_set_schedule(grid.ptr, int(s)), "lbm_set_schedule")


LBM_VARIANT_VEC16, LBM_VARIANT_SCALAR, LBM_VARIANT_VEC8, LBM_VARIANT_VEC4 = 0, 1, 2, 3
LBM_VARIANT_STAGED = 4
VARIANT_NAMES = {0: "vec16", 1: "scalar", 2: "vec8", 3: "vec4", 4: "staged"}


def lbm_set_variant(grid, variant):
    _check(load().lbm_set_variant(grid.ptr, int(variant)), "lbm_set_variant")


def lbm_set_wait_limit(grid, ns):
    """Time limit (ns) of the staged kernel's wait for its block copy; < 0 restores the default."""
    _check(load().lbm_set_wait_limit(grid.ptr, C.c_int64(int(ns))), "lbm_set_wait_limit")


def lbm_autotune(grid, n_steps):
    """Returns (chosen variant, [ms per step of each variant])."""
    chosen = C.c_int()
    ms = (C.c_double * 5)()
    _check(load().lbm_autotune(grid.ptr, int(n_steps), C.byref(chosen), ms), "lbm_autotune")
    return chosen.value, list(ms)


def lbm_set_boundary(grid, level, flags=None, bc_values=None, default_bc=None):
    fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
    bv = None if bc_values is None else np.ascontiguousarray(bc_values, dtype=np.float32)
    db = None if default_bc is None else np.ascontiguousarray(default_bc, dtype=np.float32)
    _check(load().lbm_set_boundary(
        grid.ptr, int(level), None if fl is None else C.c_void_p(fl.ctypes.data),
        None if bv is None else C.c_void_p(bv.ctypes.data),
        None if db is None else C.c_void_p(db.ctypes.data)), "lbm_set_boundary")


def lbm_init_equilibrium(grid, level, rho=None, u=None):
    pr, dr, kr = _ptr(rho, np.float64)
    pu, du, ku = _ptr(u, np.float64)
    dev = dr or du
    if rho is not None and u is not None and dr != du:
        raise ValueError("rho and u must both be host or both be device arrays")
    _check(load().lbm_init_equilibrium(grid.ptr, int(level), pr, pu, int(dev)),
           "lbm_init_equilibrium")


def lbm_step(grid, n_steps, stream=None):
    _check(load().lbm_step(grid.ptr, int(n_steps), _stream_ptr(stream)), "lbm_step")


def lbm_sync(grid):
    _check(load().lbm_sync(grid.ptr), "lbm_sync")


def _box(grid, level):
    nx, ny, nz = grid.dims
    s = 1 << level
    return nx // s, ny // s, nz // s


def lbm_get_moments(grid, level=0, rho=None, u=None):
    """Return (rho, u) as numpy arrays of shape (nz, ny, nx) and (3, nz, ny, nx),
    or fill the given CUDA tensors (device path)."""
    nx, ny, nz = _box(grid, level)
    if rho is None and u is None:
        rho = np.empty((nz, ny, nx), np.float64)
        u = np.empty((3, nz, ny, nx), np.float64)
    pr, dr, _ = _ptr(rho, np.float64)
    pu, du, _ = _ptr(u, np.float64)
    _check(load().lbm_get_moments(grid.ptr, int(level), pr, pu, int(dr or du)), "lbm_get_moments")
    return rho, u


def lbm_get_populations(grid, level, dst):
    p, d, _ = _ptr(dst, None)
    nbytes = dst.nbytes if hasattr(dst, "nbytes") else dst.numel() * dst.element_size()
    _check(load().lbm_get_populations(grid.ptr, int(level), p, nbytes, d), "lbm_get_populations")
    return dst


def lbm_set_populations(grid, level, src):
    p, d, keep = _ptr(src, None)
    nbytes = src.nbytes if hasattr(src, "nbytes") else src.numel() * src.element_size()
    _check(load().lbm_set_populations(grid.ptr, int(level), p, nbytes, d), "lbm_set_populations")


def lbm_get_populations_f64(grid, level=0, dst=None):
    nx, ny, nz = _box(grid, level)
    if dst is None:
        dst = np.empty((lbm_get_info(grid)["lattice"], nz, ny, nx), np.float64)
    p, d, _ = _ptr(dst, np.float64)
    _check(load().lbm_get_populations_f64(grid.ptr, int(level), p, d), "lbm_get_populations_f64")
    return dst


def lbm_get_layout(grid, level, what):
    n = C.c_size_t()
    lib = load()
    _check(lib.lbm_layout_bytes(grid.ptr, int(level), int(what), C.byref(n)), "lbm_layout_bytes")
    dtype = (np.uint8 if what == LBM_LAYOUT_FLAGS
             else np.uint32 if what in (LBM_LAYOUT_BOUNDARY_BITS, LBM_LAYOUT_IFACE_CROSS)
             else np.int32)
    out = np.empty(n.value // np.dtype(dtype).itemsize, dtype)
    _check(lib.lbm_get_layout(grid.ptr, int(level), int(what), C.c_void_p(out.ctypes.data),
                              n.value), "lbm_get_layout")
    return out


def lbm_conservation(grid):
    out = (C.c_double * 4)()
    _check(load().lbm_conservation(grid.ptr, out), "lbm_conservation")
    return np.array(list(out))


def lbm_conservation_noalloc(f, storage, n_voxels, flags, out, stream=None, lattice=19):
    """f, flags (or None) and out (4 float64) are contiguous CUDA tensors on
    the current device; nothing is allocated.  The sizes are checked here,
    before the pointers reach the kernels: f must hold lattice * n_voxels
    stored populations, flags n_voxels bytes and out 4 doubles."""
    import torch
    st = {"f32": 0, "f16": 1, "bf16": 2}[storage] if isinstance(storage, str) else int(storage)
    if st not in (0, 1, 2):
        raise ValueError("storage must be f32, f16 or bf16")
    q = 19 if int(lattice) == 0 else int(lattice)
    if q not in (19, 27):
        raise ValueError("lattice must be 19 or 27")
    dev = torch.cuda.current_device()
    for name, t in (("f", f), ("out", out), ("flags", flags)):
        if t is None and name == "flags":
            continue
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is not on the current device cuda:{dev}")
    n = int(n_voxels)
    if out.dtype != torch.float64 or out.numel() < 4:
        raise ValueError("out must be a float64 tensor of at least 4 elements")
    if flags is not None and (flags.dtype != torch.uint8 or flags.numel() < n):
        raise ValueError("flags must be a uint8 tensor of at least n_voxels elements")
    if n > 0 and f.numel() * f.element_size() < q * n * (4 if st == 0 else 2):
        raise ValueError(f"f holds fewer than {q} x n_voxels stored populations")
    _check(load().lbm_conservation_noalloc(
        C.c_void_p(f.data_ptr()), st, q, C.c_int64(n),
        None if flags is None else C.c_void_p(flags.data_ptr()), C.c_void_p(out.data_ptr()),
        _stream_ptr(stream)), "lbm_conservation_noalloc")


CLOSURE_PARAMS = 5313


def _dev(t):
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def lbm_closure_dataset(grid, r, tau_coarse, feats, targets):
    """feats (n_c x 16) and targets (n_c) are float32 CUDA tensors."""
    _check(load().lbm_closure_dataset(grid.ptr, int(r), float(tau_coarse), _dev(feats),
                                      _dev(targets)), "lbm_closure_dataset")


def lbm_closure_train(feats, targets, steps, batch, lr, seed, theta, stream=None):
    """Trains theta (float32 CUDA tensor, 5313) in place; returns the last loss."""
    loss = C.c_float()
    _check(load().lbm_closure_train(_dev(feats), _dev(targets), C.c_int64(targets.numel()),
                                    int(steps), int(batch), C.c_float(lr), C.c_uint64(seed),
                                    _dev(theta), C.byref(loss), _stream_ptr(stream)),
           "lbm_closure_train")
    return loss.value


def lbm_closure_grad(theta, feats, targets, idx, grad, loss, stream=None):
    _check(load().lbm_closure_grad(_dev(theta), _dev(feats), _dev(targets), _dev(idx),
                                   int(idx.numel()), _dev(grad), _dev(loss), _stream_ptr(stream)),
           "lbm_closure_grad")


def lbm_closure_forward(theta, feats, out, bf16=True, stream=None):
    _check(load().lbm_closure_forward(_dev(theta), _dev(feats), C.c_int64(out.numel()),
                                      int(bool(bf16)), _dev(out), _stream_ptr(stream)),
           "lbm_closure_forward")


def lbm_closure_load(grid, theta):
    th = np.ascontiguousarray(theta, dtype=np.float32)
    _check(load().lbm_closure_load(grid.ptr, C.c_void_p(th.ctypes.data), th.size),
           "lbm_closure_load")


class Batch:
    """Handle of lbm_batch_create; keeps the member grids alive."""

    def __init__(self, ptr, grids):
        self.ptr = ptr
        self.grids = list(grids)

    def __del__(self):
        try:
            if getattr(self, "ptr", None) and _lib is not None:
                _lib.lbm_batch_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass


def lbm_batch_create(grids):
    arr = (C.c_void_p * len(grids))(*[g.ptr.value if hasattr(g.ptr, "value") else g.ptr
                                      for g in grids])
    out = C.c_void_p()
    _check(load().lbm_batch_create(len(grids), arr, C.byref(out)), "lbm_batch_create")
    return Batch(out, grids)


def lbm_batch_destroy(batch):
    if batch.ptr:
        _check(load().lbm_batch_destroy(batch.ptr), "lbm_batch_destroy")
        batch.ptr = None


def lbm_batch_step(batch, n_steps, stream=None):
    _check(load().lbm_batch_step(batch.ptr, int(n_steps), _stream_ptr(stream)), "lbm_batch_step")


def lbm_batch_autotune(batch, n_steps):
    chosen = C.c_int()
    ms = (C.c_double * 6)()
    _check(load().lbm_batch_autotune(batch.ptr, int(n_steps), C.byref(chosen), ms),
           "lbm_batch_autotune")
    return chosen.value, list(ms)


def lbm_batch_info(batch):
    nu, ni, k = C.c_int64(), C.c_int64(), C.c_int()
    _check(load().lbm_batch_info(batch.ptr, C.byref(nu), C.byref(ni), C.byref(k)),
           "lbm_batch_info")
    return {"n_updated": nu.value, "n_items": ni.value, "ctas_per_sm": k.value}


def lbm_batch_closure_load(batch, theta, max_edge):
    """Closure on every case whose largest edge is <= max_edge (0: off)."""
    if theta is None:
        _check(load().lbm_batch_closure_load(batch.ptr, None, 0, int(max_edge)),
               "lbm_batch_closure_load")
        return
    th = np.ascontiguousarray(theta, dtype=np.float32)
    _check(load().lbm_batch_closure_load(batch.ptr, C.c_void_p(th.ctypes.data), th.size,
                                         int(max_edge)), "lbm_batch_closure_load")


def lbm_profile(grid, enable):
    _check(load().lbm_profile(grid.ptr, int(bool(enable))), "lbm_profile")


def lbm_profile_read(grid):
    stats = (lbm_kernel_stat * 32)()
    n = C.c_int()
    _check(load().lbm_profile_read(grid.ptr, stats, 32, C.byref(n)), "lbm_profile_read")
    return {stats[k].name.decode(): {"launches": stats[k].launches, "total_ms": stats[k].total_ms,
                                     "units": stats[k].units} for k in range(min(n.value, 32))}


def lbm_profile_trace(grid, max_records=100000):
    """Every recorded launch in order: (name, start_ms, end_ms, units)."""
    buf = (lbm_kernel_trace * max_records)()
    n = C.c_int()
    _check(load().lbm_profile_trace(grid.ptr, buf, max_records, C.byref(n)), "lbm_profile_trace")
    return [(buf[k].name.decode(), buf[k].start_ms, buf[k].end_ms, buf[k].units)
            for k in range(min(n.value, max_records))]
