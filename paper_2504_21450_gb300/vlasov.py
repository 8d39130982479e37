"""Python binding of the libvlgt C ABI (include/vlasov.h), argument marshalling only.

The functions keep the C names (``vl_grid_create``, ``vl_translate``, ...).  Device
memory of a grid comes from PyTorch's caching allocator through the allocator callbacks
of ``vl_device``, and work is queued on the current PyTorch CUDA stream; every step of
the computation runs in the library's CUDA kernels.  There is no CPU fallback:
``load()`` raises when the library has not been built or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

VL_OK, VL_EINVAL, VL_ENOMEM, VL_ECFL, VL_ECAPACITY, VL_ETIMEOUT, VL_ECUDA, VL_ESTATE = range(8)
VL_STORE_F32, VL_STORE_BF16_SCALED, VL_STORE_F16_SCALED = range(3)
VL_FORM_FUSED, VL_FORM_3PASS, VL_FORM_AUTO = range(3)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class vl_space_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3), ("x0", ctypes.c_double * 3)]


class vl_vmesh_desc(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int * 3), ("vmin", ctypes.c_double * 3),
                ("dv", ctypes.c_double * 3), ("block", ctypes.c_int * 3)]


class vl_device(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("device", ctypes.c_int)]


class vl_translate_opts(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("limiter", ctypes.c_int), ("ghost", ctypes.c_int),
                ("tile", ctypes.c_int * 2), ("check", ctypes.c_int), ("graph", ctypes.c_int),
                ("kernel", ctypes.c_int), ("capacity", ctypes.c_int64), ("reserved", ctypes.c_int * 4)]


class vl_step_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("blocks", ctypes.c_int64),
                ("union_blocks", ctypes.c_int64), ("dropped_blocks", ctypes.c_int64),
                ("mass", ctypes.c_double), ("dropped_mass", ctypes.c_double),
                ("mass_before", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("sweep_ms", ctypes.c_double), ("index_ms", ctypes.c_double),
                ("prune_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("capacity_regrows", ctypes.c_int64),
                ("capacity", ctypes.c_int64), ("form_used", ctypes.c_int),
                ("tile_rows_used", ctypes.c_int), ("tune_ms", ctypes.c_double * 4),
                ("updates", ctypes.c_int64), ("tail_ms", ctypes.c_double),
                ("kernel_used", ctypes.c_int), ("reserved_stats", ctypes.c_int)]


class VlError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {status_str(status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libvlgt.so.  Raises if it is missing (no silent fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libvlgt is not built ({path}); run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    p, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "vl_translate_opts_default": (None, [p]),
        "vl_grid_create": (i, [p, p, d, i, p, p]),
        "vl_grid_destroy": (i, [p]),
        "vl_set_blocks": (i, [p, i64, p, p, p, i]),
        "vl_get_block_count": (i, [p, p]),
        "vl_get_blocks": (i, [p, i64, p, p, p, i]),
        "vl_translate": (i, [p, d, ctypes.c_char_p, i, p]),
        "vl_get_block_count_window": (i, [p, p, p, p]),
        "vl_get_blocks_window": (i, [p, p, p, i64, p, p, p, i]),
        "vl_set_blocks_planes": (i, [p, i, i, i64, p, p, p, i]),
        "vl_moments": (i, [p, p, i]),
        "vl_mass": (i, [p, p]),
        "vl_stats": (i, [p, p]),
        "vl_translate_dense_noalloc": (i, [p, p, d, ctypes.c_char_p, i, p, p, p, p]),
        "vl_export": (i, [p, p, p]),
        "vl_import": (i, [p, p, ctypes.c_size_t]),
        "vl_status_str": (ctypes.c_char_p, [i]),
        "vl_last_error": (ctypes.c_char_p, [p]),
        "vl_tile_count": (i64, [p, i]),
        "vl_tile_features": (i, [p, i, p, p]),
        "vl_cost_targets": (i, [p, i, i64, i, p, p]),
        "vl_mlp_forward": (i, [p, p, i64, p, p]),
        "vl_mlp_workspace_bytes": (ctypes.c_size_t, [i64]),
        "vl_mlp_gradient": (i, [p, p, p, i64, p, ctypes.c_size_t, p, p, p]),
        "vl_mlp_train_step": (i, [p, p, p, p, p, i64, i, ctypes.c_float, p, ctypes.c_size_t, p, p]),
        "vl_mlp_capacity": (i, [p, p, i64, d, p, ctypes.c_size_t, p, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# C names, thin wrappers -------------------------------------------------------------
def status_str(st: int) -> str:
    return load().vl_status_str(st).decode()


def vl_last_error(grid) -> str:
    return load().vl_last_error(grid).decode()


def _check(st: int, where: str, grid=None):
    if st != VL_OK:
        raise VlError(st, where, vl_last_error(grid))


def vl_translate_opts_default() -> vl_translate_opts:
    o = vl_translate_opts()
    load().vl_translate_opts_default(ctypes.byref(o))
    return o


def vl_grid_create(space: vl_space_desc, vmesh: vl_vmesh_desc, threshold: float,
                   storage: int, device: vl_device | None) -> ctypes.c_void_p:
    g = ctypes.c_void_p()
    st = load().vl_grid_create(ctypes.byref(space), ctypes.byref(vmesh), float(threshold),
                               int(storage), ctypes.byref(device) if device else None,
                               ctypes.byref(g))
    _check(st, "vl_grid_create", None)
    return g


def vl_grid_destroy(grid) -> None:
    load().vl_grid_destroy(grid)


def vl_set_blocks(grid, nblocks: int, off_ptr: int, ids_ptr: int, vals_ptr: int, on_device: int):
    _check(load().vl_set_blocks(grid, nblocks, off_ptr, ids_ptr, vals_ptr, on_device),
           "vl_set_blocks", grid)


def vl_get_block_count(grid) -> int:
    n = ctypes.c_int64()
    _check(load().vl_get_block_count(grid, ctypes.byref(n)), "vl_get_block_count", grid)
    return n.value


def vl_get_blocks(grid, capacity: int, off_ptr: int, ids_ptr: int, vals_ptr: int, on_device: int):
    _check(load().vl_get_blocks(grid, capacity, off_ptr, ids_ptr, vals_ptr, on_device),
           "vl_get_blocks", grid)


def vl_get_block_count_window(grid, origin, size) -> int:
    o = (ctypes.c_int * 3)(*origin)
    sz = (ctypes.c_int * 3)(*size)
    n = ctypes.c_int64()
    _check(load().vl_get_block_count_window(grid, o, sz, ctypes.byref(n)),
           "vl_get_block_count_window", grid)
    return n.value


def vl_get_blocks_window(grid, origin, size, capacity: int, off_ptr: int, ids_ptr: int,
                         vals_ptr: int, on_device: int):
    o = (ctypes.c_int * 3)(*origin)
    sz = (ctypes.c_int * 3)(*size)
    _check(load().vl_get_blocks_window(grid, o, sz, capacity, off_ptr, ids_ptr, vals_ptr, on_device),
           "vl_get_blocks_window", grid)


def vl_set_blocks_planes(grid, z0: int, nplanes: int, nblocks: int, off_ptr: int, ids_ptr: int,
                         vals_ptr: int, on_device: int):
    _check(load().vl_set_blocks_planes(grid, int(z0), int(nplanes), int(nblocks), off_ptr, ids_ptr,
                                       vals_ptr, on_device), "vl_set_blocks_planes", grid)


def vl_translate(grid, dt: float, order: str, nsteps: int, opts: vl_translate_opts | None):
    st = load().vl_translate(grid, float(dt), order.encode(), int(nsteps),
                             ctypes.byref(opts) if opts is not None else None)
    _check(st, "vl_translate", grid)


def vl_moments(grid, out_ptr: int, on_device: int):
    _check(load().vl_moments(grid, out_ptr, on_device), "vl_moments", grid)


def vl_mass(grid) -> float:
    m = ctypes.c_double()
    _check(load().vl_mass(grid, ctypes.byref(m)), "vl_mass", grid)
    return m.value


def vl_stats(grid) -> vl_step_stats:
    s = vl_step_stats()
    _check(load().vl_stats(grid, ctypes.byref(s)), "vl_stats", grid)
    return s


def vl_translate_dense_noalloc(space: vl_space_desc, vmesh: vl_vmesh_desc, dt: float, order: str,
                               limiter: int, f_in_ptr: int, f_out_ptr: int, mass_out_ptr: int,
                               stream_ptr: int) -> int:
    """Returns the status code (no exception: the caller decides)."""
    return load().vl_translate_dense_noalloc(ctypes.byref(space), ctypes.byref(vmesh), float(dt),
                                             order.encode(), int(limiter), f_in_ptr, f_out_ptr,
                                             mass_out_ptr, stream_ptr)


# Learned cost model (device pointers as ints, streams as cudaStream_t ints) ----------
VL_MLP_NIN, VL_MLP_NHIDDEN = 8, 64
VL_MLP_NPARAM = VL_MLP_NHIDDEN * VL_MLP_NIN + VL_MLP_NHIDDEN * VL_MLP_NHIDDEN + 3 * VL_MLP_NHIDDEN + 1


def vl_tile_count(space: vl_space_desc, edge: int) -> int:
    return int(load().vl_tile_count(ctypes.byref(space), int(edge)))


def vl_tile_features(grid, edge: int, features_ptr: int, union_ptr: int) -> None:
    _check(load().vl_tile_features(grid, int(edge), features_ptr, union_ptr), "vl_tile_features", grid)


def vl_cost_targets(trace_ptr: int, nsnap: int, ntiles: int, horizon: int, targets_ptr: int,
                    stream_ptr: int) -> None:
    _check(load().vl_cost_targets(trace_ptr, int(nsnap), int(ntiles), int(horizon), targets_ptr,
                                  stream_ptr), "vl_cost_targets")


def vl_mlp_forward(params_ptr: int, x_ptr: int, n: int, y_ptr: int, stream_ptr: int) -> None:
    _check(load().vl_mlp_forward(params_ptr, x_ptr, int(n), y_ptr, stream_ptr), "vl_mlp_forward")


def vl_mlp_workspace_bytes(n: int) -> int:
    return int(load().vl_mlp_workspace_bytes(int(n)))


def vl_mlp_gradient(params_ptr, x_ptr, t_ptr, n, ws_ptr, ws_bytes, grad_ptr, loss_ptr, stream_ptr) -> None:
    _check(load().vl_mlp_gradient(params_ptr, x_ptr, t_ptr, int(n), ws_ptr, int(ws_bytes), grad_ptr,
                                  loss_ptr, stream_ptr), "vl_mlp_gradient")


def vl_mlp_train_step(params_ptr, m_ptr, v_ptr, x_ptr, t_ptr, n, step, lr, ws_ptr, ws_bytes,
                      loss_ptr, stream_ptr) -> None:
    _check(load().vl_mlp_train_step(params_ptr, m_ptr, v_ptr, x_ptr, t_ptr, int(n), int(step), float(lr),
                                    ws_ptr, int(ws_bytes), loss_ptr, stream_ptr), "vl_mlp_train_step")


def vl_mlp_capacity(params_ptr, features_ptr, ntiles, margin, ws_ptr, ws_bytes, stream_ptr) -> int:
    out = ctypes.c_int64()
    _check(load().vl_mlp_capacity(params_ptr, features_ptr, int(ntiles), float(margin), ws_ptr,
                                  int(ws_bytes), ctypes.byref(out), stream_ptr), "vl_mlp_capacity")
    return int(out.value)


# Convenience object -------------------------------------------------------------------
class Grid:
    """One phase-space grid on the current CUDA device, memory from PyTorch's allocator."""

    def __init__(self, n, nv, vmin, dv, dx=(1.0, 1.0, 1.0), threshold: float = 0.0,
                 storage: int = VL_STORE_F32, device: int | None = None, allocator=None):
        """allocator: optional callable nbytes -> device pointer (int) or None, used in
        place of PyTorch's caching allocator (its blocks are still freed through it)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libvlgt needs a CUDA device; there is no CPU fallback")
        load()
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.stream = torch.cuda.current_stream(self.device)
        self.n = tuple(int(a) for a in n)
        self.nv = tuple(int(a) for a in nv)
        self.vmin = tuple(float(a) for a in vmin)
        self.dv = tuple(float(a) for a in dv)
        self.dx = tuple(float(a) for a in dx)
        self.ncells = int(np.prod(self.n))
        dev_index = self.device
        stream = self.stream

        def _alloc(nbytes, ctx):
            try:
                if allocator is not None:
                    return allocator(int(nbytes))
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev_index, stream))
            except Exception:
                return None

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self._dev = vl_device(self._alloc_cb, self._free_cb, None,
                              ctypes.c_void_p(stream.cuda_stream), dev_index)
        space = vl_space_desc((ctypes.c_int * 3)(*self.n), (ctypes.c_double * 3)(*self.dx),
                              (ctypes.c_double * 3)(0.0, 0.0, 0.0))
        vm = vl_vmesh_desc((ctypes.c_int * 3)(*self.nv), (ctypes.c_double * 3)(*self.vmin),
                           (ctypes.c_double * 3)(*self.dv), (ctypes.c_int * 3)(4, 4, 4))
        self.space = space
        self.handle = vl_grid_create(space, vm, threshold, storage, self._dev)

    def close(self):
        if getattr(self, "handle", None):
            vl_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state transfer -------------------------------------------------------------
    def set_blocks(self, off, ids, vals):
        """off/ids/vals: numpy arrays (host copy) or torch CUDA tensors (device)."""
        t = self.torch
        if isinstance(vals, t.Tensor) and vals.is_cuda:
            off = off.to(dtype=t.int64).contiguous()
            if ids.dtype != t.int16:  # carry the uint16 bit pattern in an int16 tensor
                ids = ids.to(dtype=t.int32)
                ids = t.where(ids >= 32768, ids - 65536, ids).to(dtype=t.int16)
            ids = ids.contiguous()
            vals = vals.to(dtype=t.float32).contiguous()
            vl_set_blocks(self.handle, int(vals.numel() // 64), off.data_ptr(), ids.data_ptr(),
                          vals.data_ptr(), 1)
            return
        off = np.ascontiguousarray(off, dtype=np.int64)
        ids = np.ascontiguousarray(ids, dtype=np.uint16)
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        vl_set_blocks(self.handle, int(off[-1]), off.ctypes.data, ids.ctypes.data, vals.ctypes.data, 0)

    def block_count(self) -> int:
        return vl_get_block_count(self.handle)

    def get_blocks(self):
        m = self.block_count()
        off = np.zeros(self.ncells + 1, dtype=np.int64)
        ids = np.zeros(max(m, 1), dtype=np.uint16)
        vals = np.zeros((max(m, 1), 64), dtype=np.float32)
        vl_get_blocks(self.handle, m, off.ctypes.data, ids.ctypes.data, vals.ctypes.data, 0)
        return off, ids[:m], vals[:m]

    def get_window(self, origin, size):
        m = vl_get_block_count_window(self.handle, origin, size)
        nc = int(np.prod(size))
        off = np.zeros(nc + 1, dtype=np.int64)
        ids = np.zeros(max(m, 1), dtype=np.uint16)
        vals = np.zeros((max(m, 1), 64), dtype=np.float32)
        vl_get_blocks_window(self.handle, origin, size, m, off.ctypes.data, ids.ctypes.data,
                             vals.ctypes.data, 0)
        return off, ids[:m], vals[:m]

    def export(self) -> bytes:
        n = ctypes.c_size_t()
        _check(load().vl_export(self.handle, None, ctypes.byref(n)), "vl_export", self.handle)
        buf = ctypes.create_string_buffer(n.value)
        _check(load().vl_export(self.handle, buf, ctypes.byref(n)), "vl_export", self.handle)
        return buf.raw[: n.value]

    def import_(self, data: bytes) -> None:
        buf = ctypes.create_string_buffer(data, len(data))
        _check(load().vl_import(self.handle, buf, len(data)), "vl_import", self.handle)

    def translate(self, dt: float, order: str = "xyz", nsteps: int = 1, form: int = VL_FORM_FUSED,
                  limiter: bool = True, check: bool = False, graph: bool = False, capacity: int = 0,
                  tile_rows: int = 0, ghost: int = 3, kernel: int = 0):
        o = vl_translate_opts_default()
        o.tile[1] = int(tile_rows)
        o.kernel = int(kernel)
        o.ghost = int(ghost)
        o.form = int(form)
        o.limiter = int(bool(limiter))
        o.check = int(bool(check))
        o.graph = int(bool(graph))
        o.capacity = int(capacity)
        vl_translate(self.handle, dt, order, nsteps, o)

    def moments(self) -> np.ndarray:
        out = np.zeros((self.ncells, 7), dtype=np.float64)
        vl_moments(self.handle, out.ctypes.data, 0)
        return out

    def mass(self) -> float:
        return vl_mass(self.handle)

    def tile_features(self, edge: int = 8):
        """(features [ntiles][8], union blocks [ntiles]) as CUDA tensors."""
        t = self.torch
        nt = vl_tile_count(self.space, edge)
        f = t.empty((nt, VL_MLP_NIN), dtype=t.float32, device=self.device)
        u = t.empty(nt, dtype=t.float32, device=self.device)
        vl_tile_features(self.handle, edge, f.data_ptr(), u.data_ptr())
        return f, u

    def stats(self) -> vl_step_stats:
        return vl_stats(self.handle)
