"""The allocation-free translation step, for callers that cannot allocate device memory
(under a memory budget owned by another runtime, or without access to an allocator),
checked against the regular entry point.

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


@pytest.mark.parametrize("order, limiter", [("xyz", 1), ("xyz", 0), ("zxy", 1), ("yzx", 1)])
def test_noalloc_step_matches_regular_entry_point(order, limiter):
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
        g.translate(dt, order, 1, vlasov.VL_FORM_FUSED, limiter=bool(limiter), check=True)
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
        st = vlasov.vl_translate_dense_noalloc(space, vm, dt, order, limiter, f.data_ptr(), out.data_ptr(),
                                               mass.data_ptr(), stream.cuda_stream)
        assert st == vlasov.VL_OK, vlasov.status_str(st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref, ref_mass = want[k]
        assert np.abs(got.astype(np.float64) - ref).max() <= VAL_TOL * np.abs(ref).max()
        assert abs(float(mass.item()) - ref_mass) <= MASS_TOL * ref_mass
        f = out


def test_noalloc_rejects_what_does_not_fit():
    """One spatial cell with 65536 block ids: the per-id tables alone exceed the static
    array, while f itself is 16 MB, so the buffers passed are the full size the call
    describes."""
    import torch
    vlasov.load(build_if_missing=True)
    space = vlasov.vl_space_desc((ctypes.c_int * 3)(1, 1, 1), (ctypes.c_double * 3)(1, 1, 1),
                                 (ctypes.c_double * 3)(0, 0, 0))
    vm = vlasov.vl_vmesh_desc((ctypes.c_int * 3)(256, 256, 64), (ctypes.c_double * 3)(-128, -128, -32),
                              (ctypes.c_double * 3)(1, 1, 1), (ctypes.c_int * 3)(4, 4, 4))
    nb = 64 * 64 * 16
    f_in = torch.zeros(nb * 64, device="cuda")
    f_out = torch.zeros(nb * 64, device="cuda")
    mass = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = vlasov.vl_translate_dense_noalloc(space, vm, 1e-3, "xyz", 1, f_in.data_ptr(), f_out.data_ptr(),
                                           mass.data_ptr(), 0)
    assert st == vlasov.VL_ECAPACITY
    st = vlasov.vl_translate_dense_noalloc(space, vm, 1e-3, "xyz", 1, f_in.data_ptr(), f_in.data_ptr(),
                                           mass.data_ptr(), 0)
    assert st == vlasov.VL_EINVAL  # in and out must differ
    torch.cuda.synchronize()
    assert float(f_out.abs().max()) == 0.0  # nothing was written
