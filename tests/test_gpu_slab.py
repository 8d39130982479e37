"""The z-slab decomposition on the GPU path: several slab grids of one process (one
GPU), each a library grid of its owned planes plus 3 ghost planes on either side, refresh
their ghosts once per step through vl_get_blocks_window / vl_set_blocks_planes (Section 3:
one coalesced ghost update per step) and step with vl_translate.  Their owned planes
equal a single-domain run bit for bit, on a dense state (ghost values written into their
slots) and on a sparse one (block sets change: the layout is rebuilt)."""
import numpy as np
import pytest

import oracle
from paper_2504_21450_gb300 import inputs, slab, vlasov

from test_slab_exchange import planes_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    vlasov.load(build_if_missing=True)


@pytest.mark.parametrize("world, order, form, density, thr", [
    (2, "xyz", vlasov.VL_FORM_FUSED, 1.0, 0.0),
    (3, "zxy", vlasov.VL_FORM_FUSED, 0.35, 0.2),
    (2, "xyz", vlasov.VL_FORM_3PASS, 0.35, 0.2),
    (1, "xyz", vlasov.VL_FORM_FUSED, 0.35, 0.2),
])
def test_slabs_equal_the_single_domain_step(world, order, form, density, thr):
    n, nv = (19, 12, 14), (8, 8, 8)
    mesh = dict(nv=nv, vmin=(-4.0, -4.0, -4.0), dv=(1.0, 1.0, 1.0), dx=(1.0, 1.0, 0.8))
    init = inputs.random_blocks(n, nv, density, seed=98)
    blk = oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))
    ref = vlasov.Grid(n, nv, mesh["vmin"], mesh["dv"], mesh["dx"], threshold=thr)
    ref.set_blocks(init.off, init.ids, init.vals)
    parts = slab.slabs(n[2], world)
    grids = []
    for s in parts:
        p = planes_of(blk, n, s.origin_z, s.local_nz)
        g = vlasov.Grid((n[0], n[1], s.local_nz), nv, mesh["vmin"], mesh["dv"], mesh["dx"], threshold=thr)
        g.set_blocks(p.off, p.ids, p.vals.astype(np.float32))
        grids.append(g)
    planes = [slab.GridPlanes(g) for g in grids]
    for step in range(3):
        sends = [slab.pack(s, q.get) for s, q in zip(parts, planes)]
        for s, q, (lo, hi) in zip(parts, planes, slab.route(parts, sends)):
            slab.unpack(s, q.set, lo, hi)
        for g in grids:
            g.translate(0.15, order, 1, form, check=True)
        ref.translate(0.15, order, 1, form, check=True)
        for s, g in zip(parts, grids):
            got = g.get_window((0, 0, slab.GHOST), (n[0], n[1], s.owned))
            want = ref.get_window((0, 0, s.z0), (n[0], n[1], s.owned))
            for a, b in zip(got, want):
                np.testing.assert_array_equal(a, b, err_msg=f"step {step}, slab {s.rank}")
    for g in grids + [ref]:
        g.close()
