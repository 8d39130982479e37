"""The allocation-free translation step, for callers that cannot allocate device memory
(inside a graph capture, under a memory budget owned by another runtime, or without
access to an allocator), checked against the regular entry point.

Kept in a file of its own, collected last, so that a run stopping at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2504_21450_gb300 import inputs, vlasov

from parity import MASS_TOL, VAL_TOL

pytestmark = pytest.mark.gpu


def to_storage(off, ids, vals, ncells, nb):
    """Dense per-cell lists -> the library's storage order f[b][q][cell][16]."""
    assert np.array_equal(np.diff(off), np.full(ncells, nb))
    assert np.array_equal(ids.reshape(ncells, nb), np.tile(np.arange(nb), (ncells, 1)))
    v = np.asarray(vals, dtype=np.float32).reshape(ncells, nb, 4, 16)
    return np.ascontiguousarray(v.transpose(1, 2, 0, 3)).reshape(-1)


def test_noalloc_step_matches_regular_entry_point():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    vlasov.load(build_if_missing=True)
    n, nv = (35, 20, 12), (8, 8, 12)
    vmin, dv, dx, dt = (-4.0, -4.0, -6.0), (1.0, 1.0, 1.0), (1.0, 1.5, 1.0), 0.15
    nb = (nv[0] // 4) * (nv[1] // 4) * (nv[2] // 4)
    ncells = int(np.prod(n))
    init = inputs.random_blocks(n, nv, 1.0, seed=77)

    # regular entry point: two steps, state read back after each
    g = vlasov.Grid(n, nv, vmin, dv, dx, threshold=0.0)
    g.set_blocks(init.off, init.ids, init.vals)
    want = []
    for _ in range(2):
        g.translate(dt, "xyz", 1, vlasov.VL_FORM_FUSED, check=True)
        off, ids, vals = g.get_blocks()
        want.append((to_storage(off, ids, vals, ncells, nb), g.stats().mass))
    g.close()

    # allocation-free entry point: two calls in a row, output of the first feeds the second
    space = vlasov.vl_space_desc((ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*dx), (ctypes.c_double * 3)(0, 0, 0))
    vm = vlasov.vl_vmesh_desc((ctypes.c_int * 3)(*nv), (ctypes.c_double * 3)(*vmin),
                              (ctypes.c_double * 3)(*dv), (ctypes.c_int * 3)(4, 4, 4))
    f = torch.from_numpy(to_storage(init.off, init.ids, init.vals, ncells, nb)).cuda()
    mass = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(2):
        out = torch.empty_like(f)
        st = vlasov.vl_translate_dense_noalloc(space, vm, dt, "xyz", 1, f.data_ptr(), out.data_ptr(),
                                               mass.data_ptr(), stream.cuda_stream)
        assert st == vlasov.VL_OK, vlasov.status_str(st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref, ref_mass = want[k]
        assert np.abs(got.astype(np.float64) - ref).max() <= VAL_TOL * np.abs(ref).max()
        assert abs(float(mass.item()) - ref_mass) <= MASS_TOL * ref_mass
        f = out


def test_noalloc_rejects_what_does_not_fit():
    import torch
    vlasov.load(build_if_missing=True)
    # 4096 block ids and many tiles: the work list exceeds the static array
    space = vlasov.vl_space_desc((ctypes.c_int * 3)(256, 256, 8), (ctypes.c_double * 3)(1, 1, 1),
                                 (ctypes.c_double * 3)(0, 0, 0))
    vm = vlasov.vl_vmesh_desc((ctypes.c_int * 3)(64, 64, 64), (ctypes.c_double * 3)(-32, -32, -32),
                              (ctypes.c_double * 3)(1, 1, 1), (ctypes.c_int * 3)(4, 4, 4))
    dummy = torch.zeros(16, device="cuda")
    st = vlasov.vl_translate_dense_noalloc(space, vm, 0.01, "xyz", 1, dummy.data_ptr(),
                                           dummy.data_ptr() + 64, dummy.data_ptr(), 0)
    assert st == vlasov.VL_ECAPACITY
    st = vlasov.vl_translate_dense_noalloc(space, vm, 0.01, "xyz", 1, dummy.data_ptr(),
                                           dummy.data_ptr(), dummy.data_ptr(), 0)
    assert st == vlasov.VL_EINVAL  # in and out must differ
