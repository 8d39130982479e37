"""FP64 CPU oracle of the coalesced-ghost Vlasov translation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA path: the arithmetic lives in
``vlref.c`` (plain loops, IEEE double, no floating-point contraction), and this module
only compiles it with gcc and marshals numpy arrays through ctypes.

Sparse phase-space state is passed around as a ``Blocks`` triple that mirrors the
library's transfer format: ``off`` (int64, ncells+1 offsets), ``ids`` (uint16 block ids,
sorted per cell) and ``vals`` (float64, 64 values per block, vx fastest).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlref.c")
_HDR = os.path.join(_HERE, "vlref.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libvlref.so")
_lib = None

AXES = {"x": 0, "y": 1, "z": 2}


def build(force: bool = False) -> str:
    """Compile vlref.c into oracle/_build/libvlref.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)
             or os.path.getmtime(_SO) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.vlref_face.restype = d
        L.vlref_face.argtypes = [d, d, d, d, i]
        L.vlref_limit.restype = None
        L.vlref_limit.argtypes = [d, p, p]
        L.vlref_outflow.restype = d
        L.vlref_outflow.argtypes = [d, d, d, d]
        L.vlref_sweep_line.argtypes = [i, i, p, p, d, i]
        L.vlref_sweep_field.argtypes = [p, i, p, p, i, d, i]
        L.vlref_step_field.argtypes = [p, i, p, p, p, i]
        L.vlref_step_field_gt.argtypes = [p, p, p, p, i, i, p]
        L.vlref_gt_regions.restype = None
        L.vlref_gt_regions.argtypes = [p, i, p, p, p]
        L.vlref_union.argtypes = [p, i, ctypes.c_int64, p, p, p, p]
        L.vlref_translate.argtypes = [p, i, p, p, p, p, d, p, i, i, p, p, p, p, p, p, p, p, i]
        L.vlref_prune.argtypes = [ctypes.c_int64, p, d, d, p, p]
        L.vlref_mass.restype = d
        L.vlref_mass.argtypes = [ctypes.c_int64, p, d]
        L.vlref_moments.argtypes = [ctypes.c_int64, p, p, p, p, p, p, p]
        L.vlref_max_threads.restype = i
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    # data_as keeps a reference to the array for as long as the pointer object lives,
    # so temporaries passed straight into a call stay valid during it
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc == 2:
        raise ValueError(f"{what}: Courant number above 1 (|v_d| dt / dx_d > 1)")
    if rc != 0:
        raise ValueError(f"{what}: bad argument (code {rc})")


def _ivec(v, dtype=np.int32) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=dtype))


def order_of(order: str) -> np.ndarray:
    """'xyz' -> [0, 1, 2]; any permutation of the three axes."""
    o = [AXES[ch] for ch in order]
    if sorted(o) != [0, 1, 2]:
        raise ValueError(f"sweep order must be a permutation of 'xyz', got {order!r}")
    return _ivec(o)


# ---------------------------------------------------------------- PPM pieces
def face(am1: float, a0: float, a1: float, a2: float, limiter: bool = True) -> float:
    return lib().vlref_face(am1, a0, a1, a2, int(limiter))


def limit(a: float, aL: float, aR: float) -> tuple[float, float]:
    l, r = ctypes.c_double(aL), ctypes.c_double(aR)
    lib().vlref_limit(a, ctypes.byref(l), ctypes.byref(r))
    return l.value, r.value


def outflow(aL: float, a: float, aR: float, c: float) -> float:
    return lib().vlref_outflow(aL, a, aR, c)


def sweep_line(a, c: float, limiter: bool = True, periodic: bool = True) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty_like(a)
    _check(lib().vlref_sweep_line(a.size, int(periodic), _ptr(a), _ptr(out), c, int(limiter)),
           "sweep_line")
    return out


# ---------------------------------------------------------------- scalar fields
# Fields are numpy arrays of shape (nz, ny, nx): cell index x + nx*(y + ny*z).
def _dims(f: np.ndarray) -> np.ndarray:
    return _ivec([f.shape[2], f.shape[1], f.shape[0]])


def sweep_field(f, dim: int, c: float, limiter: bool = True, periodic: bool = True) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _check(lib().vlref_sweep_field(_ptr(_dims(f)), int(periodic), _ptr(f), _ptr(out), dim, c,
                                   int(limiter)), "sweep_field")
    return out


def step_field(f, c, order: str = "xyz", limiter: bool = True, periodic: bool = True) -> np.ndarray:
    out = np.array(f, dtype=np.float64, order="C", copy=True)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    _check(lib().vlref_step_field(_ptr(_dims(out)), int(periodic), _ptr(out), _ptr(cc),
                                  _ptr(order_of(order)), int(limiter)), "step_field")
    return out


def step_field_gt(f, c, order: str = "xyz", limiter: bool = True, k: int = 3,
                  box=(4, 4, 4)) -> np.ndarray:
    """GT-k tiled step (Section 3.2) with boxes of extents box (x, y, z); an extent of 0
    makes the boxes span that whole periodic axis, with no ghost layer along it."""
    out = np.array(f, dtype=np.float64, order="C", copy=True)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    _check(lib().vlref_step_field_gt(_ptr(_dims(out)), _ptr(out), _ptr(cc),
                                     _ptr(order_of(order)), int(limiter), int(k),
                                     _ptr(_ivec(box))), "step_field_gt")
    return out


# ---------------------------------------------------------------- Section 3 regions
def gt_regions(local, k: int, order: str = "xyz") -> tuple[np.ndarray, np.ndarray]:
    """Volumes of active_j and source_j (j = sweep index) for a box of extents local."""
    loc = np.ascontiguousarray(local, dtype=np.float64)
    act = np.zeros(3)
    src = np.zeros(3)
    lib().vlref_gt_regions(_ptr(loc), int(k), _ptr(order_of(order)), _ptr(act), _ptr(src))
    return act, src


def gt_ratios(edge: float, k: int, order: str = "xyz") -> tuple[float, float]:
    """Active and source cell ratios of an ideal periodic cubic domain (Section 3.3).

    Reading of the denominators: the classical solver computes on the local cells once
    per direction (3 L^3 in total) and its per-direction ghost update covers the local
    cells widened by the 2-cell stencil of their face neighbours, i.e. +-3 cells along
    the sweep (3 L^2 (L+6) in total)."""
    act, src = gt_regions([edge] * 3, k, order)
    return float(act.sum() / (3 * edge ** 3)), float(src.sum() / (3 * edge ** 2 * (edge + 6)))


# ---------------------------------------------------------------- sparse phase space
@dataclass
class Blocks:
    off: np.ndarray   # int64 [ncells+1]
    ids: np.ndarray   # uint16 [nblocks]
    vals: np.ndarray  # float64 [nblocks, 64]

    @property
    def nblocks(self) -> int:
        return int(self.off[-1])

    def copy(self) -> "Blocks":
        return Blocks(self.off.copy(), self.ids.copy(), self.vals.copy())


def as_blocks(off, ids, vals) -> Blocks:
    return Blocks(np.ascontiguousarray(off, dtype=np.int64),
                  np.ascontiguousarray(ids, dtype=np.uint16),
                  np.ascontiguousarray(np.asarray(vals, dtype=np.float64).reshape(-1, 64)))


def union(n, nb: int, blk: Blocks, periodic: bool = True) -> tuple[np.ndarray, np.ndarray]:
    nn = _ivec(n)
    ncell = int(np.prod(n))
    off_u = np.zeros(ncell + 1, dtype=np.int64)
    _check(lib().vlref_union(_ptr(nn), int(periodic), nb, _ptr(blk.off), _ptr(blk.ids),
                             _ptr(off_u), None), "union")
    ids_u = np.zeros(max(int(off_u[-1]), 1), dtype=np.uint16)
    _check(lib().vlref_union(_ptr(nn), int(periodic), nb, _ptr(blk.off), _ptr(blk.ids),
                             _ptr(off_u), _ptr(ids_u)), "union")
    return off_u, ids_u[: int(off_u[-1])]


@dataclass
class Mesh:
    """Spatial box and velocity mesh (block size 4x4x4)."""
    n: tuple            # (nx, ny, nz)
    nv: tuple           # velocity cells per dimension (multiples of 4)
    vmin: tuple
    dv: tuple
    dx: tuple = (1.0, 1.0, 1.0)
    periodic: bool = True

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))

    @property
    def nb(self) -> int:
        return int(np.prod([v // 4 for v in self.nv]))

    @property
    def phase_cell_volume(self) -> float:
        return float(np.prod(self.dx) * np.prod(self.dv))


def translate(mesh: Mesh, blk: Blocks, dt: float, order: str = "xyz", limiter: bool = True,
              gt_k: int = 0, gt_box=(4, 4, 4), nthreads: int = 0) -> tuple[Blocks, float]:
    """One step into the union layout; returns (union blocks with new values, leaked)."""
    off_u, ids_u = union(mesh.n, mesh.nb, blk, mesh.periodic)
    vals_u = np.zeros((int(off_u[-1]), 64))
    leaked = ctypes.c_double(0.0)
    rc = lib().vlref_translate(
        _ptr(_ivec(mesh.n)), int(mesh.periodic), _ptr(_ivec(mesh.dx, np.float64)),
        _ptr(_ivec(mesh.nv)), _ptr(_ivec(mesh.vmin, np.float64)),
        _ptr(_ivec(mesh.dv, np.float64)), float(dt), _ptr(order_of(order)), int(limiter),
        int(gt_k), _ptr(_ivec(gt_box)), _ptr(blk.off), _ptr(blk.ids), _ptr(blk.vals),
        _ptr(off_u), _ptr(ids_u), _ptr(vals_u), ctypes.byref(leaked), int(nthreads))
    _check(rc, "translate")
    return Blocks(off_u, ids_u, vals_u), leaked.value


def prune(mesh: Mesh, blk: Blocks, threshold: float) -> tuple[Blocks, np.ndarray, float]:
    """Apply the sparsity rule; returns (kept blocks, keep flags, dropped mass)."""
    keep = np.zeros(blk.nblocks, dtype=np.uint8)
    dropped = ctypes.c_double(0.0)
    _check(lib().vlref_prune(blk.nblocks, _ptr(blk.vals), float(threshold),
                             mesh.phase_cell_volume, _ptr(keep), ctypes.byref(dropped)), "prune")
    k = keep.astype(bool)
    cell_of = np.repeat(np.arange(mesh.ncells), np.diff(blk.off))
    counts = np.bincount(cell_of[k], minlength=mesh.ncells)
    off = np.zeros(mesh.ncells + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return Blocks(off, np.ascontiguousarray(blk.ids[k]), np.ascontiguousarray(blk.vals[k])), keep, dropped.value


@dataclass
class StepStats:
    union_blocks: int
    kept_blocks: int
    dropped_mass: float
    leaked: float


def step(mesh: Mesh, blk: Blocks, dt: float, threshold: float, order: str = "xyz",
         limiter: bool = True, gt_k: int = 0, gt_box=(4, 4, 4), nthreads: int = 0):
    """Union -> three shears -> sparsity rule: one full step of the sparse phase space."""
    u, leaked = translate(mesh, blk, dt, order, limiter, gt_k, gt_box, nthreads)
    kept, keep, dropped = prune(mesh, u, threshold)
    return kept, StepStats(u.nblocks, kept.nblocks, dropped, leaked), u, keep


def mass(mesh: Mesh, blk: Blocks) -> float:
    return lib().vlref_mass(blk.nblocks, _ptr(blk.vals), mesh.phase_cell_volume)


def moments(mesh: Mesh, blk: Blocks) -> np.ndarray:
    out = np.zeros((mesh.ncells, 7))
    _check(lib().vlref_moments(mesh.ncells, _ptr(_ivec(mesh.nv)),
                               _ptr(_ivec(mesh.vmin, np.float64)),
                               _ptr(_ivec(mesh.dv, np.float64)), _ptr(blk.off), _ptr(blk.ids),
                               _ptr(blk.vals), _ptr(out)), "moments")
    return out


def max_threads() -> int:
    return lib().vlref_max_threads()
