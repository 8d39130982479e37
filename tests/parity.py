"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and the FP64
oracle on the same seeded inputs and compare block sets, values and mass."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2504_21450_gb300 import vlasov

# Acceptance of the CUDA path against the FP64 oracle (FP32 storage):
# values within max-abs 1e-5 * max f, total mass within 1e-6 relative, block sets equal
# except blocks whose oracle maximum lies within a relative 1e-5 of the threshold.
VAL_TOL = 1e-5
MASS_TOL = 1e-6
GUARD = 1e-5


def gpu_grid(mesh: oracle.Mesh, threshold: float) -> vlasov.Grid:
    return vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, threshold=threshold)


def block_keys(off, ids):
    """(cell, id) of every block as one sorted int64 key cell * 65536 + id."""
    off = np.asarray(off)
    cell = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    return cell * 65536 + np.asarray(ids, dtype=np.int64), cell


def compare_step(mesh, before: oracle.Blocks, gpu_after, threshold, dt, order="xyz",
                 limiter=True, cells=None, gt_k=0, gt_box=(4, 4, 4)):
    """One oracle step from `before`, compared with the GPU's result (off, ids, vals).
    `cells` restricts the comparison to a subset of cell indices (windowed parity);
    gt_k > 0 takes the oracle's tiled GT-k step with boxes gt_box.
    Returns (max abs error, max |f| of the oracle, ambiguous blocks, oracle blocks, stats)."""
    ref, st, u, keep = oracle.step(mesh, before, dt, threshold, order, limiter, gt_k, gt_box)
    if limiter:
        assert st.leaked == 0.0
    off, ids, vals = gpu_after
    rk, rc = block_keys(ref.off, ref.ids)
    gk, gc = block_keys(off, ids)
    uk, uc = block_keys(u.off, u.ids)
    amb = np.zeros(0, dtype=np.int64)
    if threshold > 0:
        near = np.abs(u.vals.max(axis=1) - threshold) <= GUARD * threshold
        amb = uk[near]
    rsel = ~np.isin(rk, amb)
    gsel = ~np.isin(gk, amb)
    if cells is not None:
        cells = np.asarray(cells, dtype=np.int64)
        rsel &= np.isin(rc, cells)
        gsel &= np.isin(gc, cells)
        amb = amb[np.isin(amb // 65536, cells)]
    r_keys, g_keys = rk[rsel], gk[gsel]
    if not np.array_equal(r_keys, g_keys):
        only_r = np.setdiff1d(r_keys, g_keys)[:5]
        only_g = np.setdiff1d(g_keys, r_keys)[:5]
        raise AssertionError(f"block sets differ: only oracle {[(k >> 16, k & 65535) for k in only_r]}, "
                             f"only GPU {[(k >> 16, k & 65535) for k in only_g]}")
    rv = ref.vals[rsel]
    gv = np.asarray(vals)[gsel].astype(np.float64)
    fmax = float(np.abs(rv).max()) if rv.size else 0.0
    err = float(np.abs(gv - rv).max()) if rv.size else 0.0
    return err, fmax, int(amb.size), ref, st
