"""GPU parity of the plane-batched GT3 kernel (fused form, `kernel` option 1) through the
C ABI: bit for bit against the classical 3-pass form (both walk every line from its
upwind end with the same arithmetic, Section 3: Ghost Translation gives correct data in
the local domain), and against the FP64 oracle step by step, on dense and sparse states
with ragged tiles, every sweep order the kernel takes, the limiter on and off."""
import numpy as np
import pytest

import oracle
from paper_2504_21450_gb300 import inputs, vlasov

from parity import VAL_TOL, MASS_TOL, compare_step, gpu_grid

pytestmark = pytest.mark.gpu

BATCHED, ROWS = 1, 2
ORDERS = ["xyz", "yxz", "xzy", "zxy"]   # streamed axis z or y; sweep 0 along x or not


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    vlasov.load(build_if_missing=True)
    oracle.build()


def as_ref(init):
    return oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))


def run(mesh, init, thr, dt, order, steps, form, kernel=0, limiter=True, graph=False):
    g = gpu_grid(mesh, thr)
    g.set_blocks(init.off, init.ids, init.vals)
    g.translate(dt, order, steps, form, limiter=limiter, check=True, kernel=kernel, graph=graph)
    s = g.stats()
    out = g.get_blocks()
    g.close()
    return out, s


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("n", [(37, 19, 11), (8, 8, 8), (5, 3, 17)])
def test_batched_equals_3pass_bit_for_bit(order, n):
    """Dense and sparse blocks, pruning, ragged tiles and halos that wrap a short axis
    several times: two steps give the 3-pass form's state bit for bit."""
    init = inputs.random_blocks(n, (8, 8, 8), 0.35, seed=90)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0, -4.0, -4.0), dv=(1.0, 1.0, 1.0), dx=(1.0, 1.2, 0.9))
    a, sa = run(mesh, init, 0.05, 0.2, order, 2, vlasov.VL_FORM_FUSED, BATCHED)
    b, _ = run(mesh, init, 0.05, 0.2, order, 2, vlasov.VL_FORM_3PASS)
    assert sa.kernel_used == BATCHED and sa.tile_rows_used == 16
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("order", ["xyz", "zxy"])
def test_batched_sparse_steps_against_oracle(order):
    """Sparse state with the sparsity rule removing blocks: each GPU step against one
    oracle step from the GPU's previous state; dropped mass and total mass too."""
    n = (37, 19, 11)
    init = inputs.random_blocks(n, (8, 8, 8), 0.25, seed=91)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0, -4.0, -5.0), dv=(1.0, 1.0, 1.25), dx=(1.0, 1.0, 1.5))
    thr = 0.3
    g = gpu_grid(mesh, thr)
    g.set_blocks(init.off, init.ids, init.vals)
    before = as_ref(init)
    for step in range(3):
        g.translate(0.15, order, 1, vlasov.VL_FORM_FUSED, check=True, kernel=BATCHED)
        after = g.get_blocks()
        err, fmax, amb, ref, st = compare_step(mesh, before, after, thr, 0.15, order)
        assert err <= VAL_TOL * fmax, (step, err, fmax)
        assert st.kept_blocks < st.union_blocks
        s = g.stats()
        assert s.kernel_used == BATCHED
        assert abs(s.dropped_mass - st.dropped_mass) <= 1e-5 * max(st.dropped_mass, 1e-30)
        m_ref = oracle.mass(mesh, ref)
        assert abs(s.mass - m_ref) <= MASS_TOL * m_ref
        before = oracle.as_blocks(*[np.asarray(x) for x in after[:2]], after[2].astype(np.float64))
    g.close()


@pytest.mark.parametrize("order", ["xyz", "yxz"])
def test_batched_limiter_off_dense(order):
    n = (20, 18, 7)
    init = inputs.random_blocks(n, (8, 4, 4), 1.0, seed=92, positive=False)
    mesh = oracle.Mesh(n=n, nv=(8, 4, 4), vmin=(-4.0, 0.0, -4.0), dv=(1.0,) * 3)
    got, s = run(mesh, init, 0.0, 0.2, order, 1, vlasov.VL_FORM_FUSED, BATCHED, limiter=False)
    assert s.kernel_used == BATCHED
    ref, _ = oracle.translate(mesh, as_ref(init), 0.2, order, limiter=False)
    np.testing.assert_array_equal(got[0], ref.off)
    assert np.abs(got[2] - ref.vals).max() <= VAL_TOL * np.abs(ref.vals).max()
    three, _ = run(mesh, init, 0.0, 0.2, order, 1, vlasov.VL_FORM_3PASS, limiter=False)
    np.testing.assert_array_equal(got[2], three[2])


def test_batched_uniform_config_window():
    """The 32x32x8 grid with the uniform workload's distributions (full 32^3 velocity
    mesh, 5% density noise): one step against the oracle over the whole grid."""
    import dataclasses
    cfg = dataclasses.replace(inputs.CONFIGS["uniform"], n=(32, 32, 8))
    init = inputs.generate(cfg)
    mesh = oracle.Mesh(n=cfg.n, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx)
    g = gpu_grid(mesh, init.threshold)
    g.set_blocks(init.off, init.ids, init.vals)
    g.translate(cfg.dt, "xyz", 1, vlasov.VL_FORM_FUSED, check=True, kernel=BATCHED)
    err, fmax, amb, ref, _ = compare_step(mesh, as_ref(init), g.get_blocks(), init.threshold, cfg.dt)
    assert amb == 0 and err <= VAL_TOL * fmax, (err, fmax)
    m_ref = oracle.mass(mesh, ref)
    assert abs(g.mass() - m_ref) <= MASS_TOL * m_ref
    g.close()


def test_batched_captured_steps_equal_step_by_step():
    n = (40, 33, 18)
    init = inputs.random_blocks(n, (8, 8, 8), 0.3, seed=93)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    a, _ = run(mesh, init, 0.1, 0.2, "xyz", 4, vlasov.VL_FORM_FUSED, BATCHED)
    b, sb = run(mesh, init, 0.1, 0.2, "xyz", 4, vlasov.VL_FORM_FUSED, BATCHED, graph=True)
    assert sb.graph_replays >= 1 and sb.kernel_used == BATCHED
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_default_kernel_and_where_it_does_not_apply():
    """The default fused kernel is the plane-batched one where it applies; blocks that
    straddle v = 0 or an x-last order fall back to the row-segment kernel, and asking
    for the plane-batched kernel there is VL_EINVAL."""
    n = (21, 14, 9)
    init = inputs.random_blocks(n, (8, 8, 8), 0.4, seed=94)
    ok = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    _, s = run(ok, init, 0.1, 0.2, "xyz", 1, vlasov.VL_FORM_FUSED)
    assert s.kernel_used == BATCHED
    _, s = run(ok, init, 0.1, 0.2, "yzx", 1, vlasov.VL_FORM_FUSED)
    assert s.kernel_used == ROWS
    _, s = run(ok, init, 0.1, 0.2, "xyz", 1, vlasov.VL_FORM_FUSED, ROWS)
    assert s.kernel_used == ROWS
    straddle = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-3.0, -4.0, -4.0), dv=(1.0,) * 3)
    _, s = run(straddle, init, 0.1, 0.2, "xyz", 1, vlasov.VL_FORM_FUSED)
    assert s.kernel_used == ROWS
    for mesh, order in ((straddle, "xyz"), (ok, "zyx")):
        g = gpu_grid(mesh, 0.1)
        g.set_blocks(init.off, init.ids, init.vals)
        with pytest.raises(vlasov.VlError) as e:
            g.translate(0.2, order, 1, vlasov.VL_FORM_FUSED, kernel=BATCHED)
        assert e.value.status == vlasov.VL_EINVAL
        g.close()


@pytest.mark.parametrize("storage", [vlasov.VL_STORE_BF16_SCALED, vlasov.VL_STORE_F16_SCALED])
@pytest.mark.parametrize("order", ["xyz", "yxz"])
def test_batched_16bit_storage_equals_row_segment_kernel(storage, order):
    """Scaled 16-bit storage: both fused kernels decode the stored codes, run the same
    per-velocity-cell arithmetic in FP32 and round once per step, each chunk with the
    scale of its own new values, so their states, codes included, agree bit for bit;
    sparse blocks and pruning."""
    n = (37, 19, 11)
    init = inputs.random_blocks(n, (8, 8, 8), 0.35, seed=96)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    outs = []
    for kernel in (BATCHED, ROWS):
        g = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, threshold=0.05, storage=storage)
        g.set_blocks(init.off, init.ids, init.vals)
        g.translate(0.2, order, 2, vlasov.VL_FORM_FUSED, check=True, kernel=kernel,
                    tile_rows=0 if kernel == BATCHED else 16)
        assert g.stats().kernel_used == kernel
        outs.append((g.get_blocks(), g.export()))
        g.close()
    for x, y in zip(outs[0][0], outs[1][0]):
        np.testing.assert_array_equal(x, y)
    assert outs[0][1] == outs[1][1]  # checkpoints
