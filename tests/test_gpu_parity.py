"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs -- fused (Ghost Translation) and 3-pass (classical) forms."""
import numpy as np
import pytest

import oracle
from paper_2504_21450_gb300 import inputs, vlasov

from parity import GUARD, MASS_TOL, VAL_TOL, compare_step, gpu_grid

pytestmark = pytest.mark.gpu

FORMS = {"fused": vlasov.VL_FORM_FUSED, "3pass": vlasov.VL_FORM_3PASS}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    vlasov.load(build_if_missing=True)
    oracle.build()


def as_ref(init):
    return oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))


def mesh_of(cfg, n=None):
    return oracle.Mesh(n=tuple(n or cfg.n), nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx)


@pytest.mark.parametrize("form", ["fused", "3pass"])
def test_tiny_config_matches_oracle(form):
    cfg = inputs.CONFIGS["tiny"]
    init = inputs.generate(cfg)
    mesh = mesh_of(cfg)
    g = gpu_grid(mesh, init.threshold)
    g.set_blocks(init.off, init.ids, init.vals)
    m0 = g.mass()
    g.translate(cfg.dt, "xyz", 1, FORMS[form], check=True)
    after = g.get_blocks()
    err, fmax, amb, ref, st = compare_step(mesh, as_ref(init), after, init.threshold, cfg.dt)
    assert amb == 0
    assert err <= VAL_TOL * fmax, (err, fmax)
    m_ref = oracle.mass(mesh, ref)
    assert abs(g.mass() - m_ref) <= MASS_TOL * m_ref
    assert abs(g.stats().mass - m_ref) <= MASS_TOL * m_ref
    assert abs(m0 - oracle.mass(mesh, as_ref(init))) <= 1e-12 * m_ref


def run_forms(mesh, init, dt, order, steps, limiter=True):
    out = {}
    for name, form in FORMS.items():
        g = gpu_grid(mesh, init.threshold)
        g.set_blocks(init.off, init.ids, init.vals)
        g.translate(dt, order, steps, form, limiter=limiter, check=True)
        out[name] = g.get_blocks()
        g.close()
    return out


@pytest.mark.parametrize("order", ["xyz", "yxz"])
def test_fused_equals_3pass_bit_for_bit(order):
    """Ghost Translation computes the same floating-point operations per cell as the
    classical form (Section 3: the result is correct data in the local domain): with
    the streamed axis along the velocity chunk's own axis every sweep of both forms
    walks each line from its upwind end with identical arithmetic."""
    init = inputs.random_blocks((37, 19, 11), (8, 8, 8), 0.3, seed=40)
    mesh = oracle.Mesh(n=(37, 19, 11), nv=(8, 8, 8), vmin=(-4.0, -3.0, -4.5), dv=(1.0,) * 3)
    init.threshold = 0.05
    out = run_forms(mesh, init, 0.2, order, 2)
    for a, b in zip(out["fused"], out["3pass"]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("order", ["zxy", "yzx", "xzy"])
def test_fused_matches_3pass_other_orders(order):
    """Orders whose streamed axis is not the velocity chunk's own axis use the
    sign-generic window for the streamed sweep: same result up to FP32 rounding."""
    init = inputs.random_blocks((37, 19, 11), (8, 8, 8), 0.3, seed=46)
    mesh = oracle.Mesh(n=(37, 19, 11), nv=(8, 8, 8), vmin=(-4.0, -3.0, -4.5), dv=(1.0,) * 3)
    init.threshold = 0.0
    out = run_forms(mesh, init, 0.2, order, 2)
    np.testing.assert_array_equal(out["fused"][0], out["3pass"][0])
    np.testing.assert_array_equal(out["fused"][1], out["3pass"][1])
    assert np.abs(out["fused"][2] - out["3pass"][2]).max() <= 1e-6 * np.abs(out["3pass"][2]).max()


@pytest.mark.parametrize("form", ["fused", "3pass"])
@pytest.mark.parametrize("order", ["xyz", "zxy"])
def test_sparse_ragged_tiles_step_by_step(form, order):
    """Several tiles with ragged tails, sparse blocks, pruning: each GPU step is checked
    against one oracle step started from the GPU's own previous state."""
    n = (37, 19, 11)
    init = inputs.random_blocks(n, (8, 8, 12), 0.25, seed=41)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 12), vmin=(-4.0, -4.0, -6.0), dv=(1.0,) * 3, dx=(1.0, 1.0, 1.5))
    thr = 0.3
    g = gpu_grid(mesh, thr)
    g.set_blocks(init.off, init.ids, init.vals)
    before = as_ref(init)
    for step in range(3):
        g.translate(0.15, order, 1, FORMS[form], check=True)
        after = g.get_blocks()
        err, fmax, amb, ref, st = compare_step(mesh, before, after, thr, 0.15, order)
        assert err <= VAL_TOL * fmax, (step, err, fmax)
        assert st.kept_blocks < st.union_blocks  # the sparsity rule removed blocks
        s = g.stats()
        assert abs(s.dropped_mass - st.dropped_mass) <= 1e-5 * max(st.dropped_mass, 1e-30)
        before = oracle.as_blocks(*[np.asarray(a) for a in after[:2]], after[2].astype(np.float64))


def test_limiter_off_dense():
    n = (20, 9, 7)
    init = inputs.random_blocks(n, (8, 4, 4), 1.0, seed=42, positive=False)
    mesh = oracle.Mesh(n=n, nv=(8, 4, 4), vmin=(-4.0, -2.0, -2.0), dv=(1.0,) * 3)
    for name, form in FORMS.items():
        g = gpu_grid(mesh, 0.0)
        g.set_blocks(init.off, init.ids, init.vals)
        g.translate(0.2, "yxz", 1, form, limiter=False, check=True)
        ref, _ = oracle.translate(mesh, as_ref(init), 0.2, "yxz", limiter=False)
        off, ids, vals = g.get_blocks()
        np.testing.assert_array_equal(off, ref.off)
        assert np.abs(vals - ref.vals).max() <= VAL_TOL * np.abs(ref.vals).max()


def test_whole_cell_shift_at_unit_courant():
    n = (6, 5, 4)
    mesh = oracle.Mesh(n=n, nv=(4, 4, 4), vmin=(-2.0,) * 3, dv=(1.0,) * 3, dx=(1.5,) * 3)
    rng = np.random.default_rng(43)
    ncell = int(np.prod(n))
    vals = rng.uniform(0.1, 1.0, (ncell, 64)).astype(np.float32)
    for form in FORMS.values():
        g = gpu_grid(mesh, 0.0)
        g.set_blocks(np.arange(ncell + 1), np.zeros(ncell, np.uint16), vals)
        g.translate(1.0, "zxy", 1, form, check=True)
        _, _, out = g.get_blocks()
        for v in (0, 3, 12, 15, 48, 51, 60, 63):
            iv = (v % 4, (v // 4) % 4, v // 16)
            s = [1 if i == 3 else -1 for i in iv]
            want = np.roll(vals[:, v].reshape(n[2], n[1], n[0]), (s[2], s[1], s[0]), axis=(0, 1, 2))
            np.testing.assert_allclose(out[:, v].reshape(n[2], n[1], n[0]), want, rtol=3e-7)


@pytest.mark.parametrize("n", [(1, 1, 1), (1, 2, 3), (3, 1, 70), (65, 2, 1), (130, 3, 2)])
def test_degenerate_and_wide_grids(n):
    init = inputs.random_blocks(n, (8, 8, 8), 0.5, seed=44)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    for form in FORMS.values():
        g = gpu_grid(mesh, 0.1)
        g.set_blocks(init.off, init.ids, init.vals)
        g.translate(0.2, "xzy", 1, form, check=True)
        err, fmax, amb, _, _ = compare_step(mesh, as_ref(init), g.get_blocks(), 0.1, 0.2, "xzy")
        assert err <= VAL_TOL * fmax


def test_empty_state_and_errors():
    mesh = oracle.Mesh(n=(4, 4, 4), nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    g = gpu_grid(mesh, 0.0)
    with pytest.raises(vlasov.VlError) as e:
        g.translate(0.1)
    assert e.value.status == vlasov.VL_ESTATE
    g.set_blocks(np.zeros(65, np.int64), np.zeros(0, np.uint16), np.zeros((0, 64), np.float32))
    g.translate(0.1, "xyz", 2, check=True)
    assert g.block_count() == 0
    with pytest.raises(vlasov.VlError) as e:
        g.translate(0.3)  # |v| = 3.5 -> c = 1.05
    assert e.value.status == vlasov.VL_ECFL
    with pytest.raises(vlasov.VlError) as e:
        g.translate(0.1, "xxy")
    assert e.value.status == vlasov.VL_EINVAL
    off = np.zeros(65, np.int64)
    off[1:] = 2
    with pytest.raises(vlasov.VlError) as e:
        g.set_blocks(off, np.array([3, 1], np.uint16), np.zeros((2, 64), np.float32))
    assert e.value.status == vlasov.VL_EINVAL
    with pytest.raises(vlasov.VlError) as e:
        g.set_blocks(off, np.array([1, 99], np.uint16), np.zeros((2, 64), np.float32))
    assert e.value.status == vlasov.VL_EINVAL


def test_mass_conservation_and_moments():
    n = (12, 10, 8)
    init = inputs.random_blocks(n, (8, 8, 8), 0.6, seed=45)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(0.5, 1.0, 1.0), dx=(1.0, 2.0, 1.0))
    g = gpu_grid(mesh, 0.0)
    g.set_blocks(init.off, init.ids, init.vals)
    m0 = g.mass()
    np.testing.assert_allclose(g.moments(), oracle.moments(mesh, as_ref(init)), rtol=1e-11, atol=1e-13)
    g.translate(0.1, "xyz", 5, check=True)
    assert abs(g.mass() - m0) <= MASS_TOL * m0
    s = g.stats()
    assert 0.0 < s.tail_ms < s.sweep_ms  # the persistent kernel's idle tail, fused steps
    assert s.steps == 5 and s.dropped_blocks == 0 and abs(s.mass - m0) <= MASS_TOL * m0


@pytest.mark.parametrize("form", ["fused", "3pass"])
def test_uniform_config_full_size_window(form):
    """The 64^3 x 32^3 workload at full size, in the configuration the benchmark times:
    a 16^3 window of the state is read before and after one step, and the oracle
    recomputes the 10^3 interior (dependence radius 3 per step) from the window."""
    import torch
    cfg = inputs.CONFIGS["uniform"]
    off, ids, vals, thr = inputs.generate_torch(cfg, "cuda")
    mesh = mesh_of(cfg)
    g = gpu_grid(mesh, thr)
    g.set_blocks(off, ids, vals)
    del off, ids, vals
    torch.cuda.empty_cache()
    origin, size = (55, 7, 60), (16, 16, 16)  # wraps around x and z
    pre = g.get_window(origin, size)
    g.translate(cfg.dt, "xyz", 1, FORMS[form], check=True)
    post = g.get_window(origin, size)
    wmesh = oracle.Mesh(n=size, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx, periodic=False)
    inner = [x + size[0] * (y + size[1] * z) for z in range(3, 13) for y in range(3, 13) for x in range(3, 13)]
    err, fmax, amb, _, _ = compare_step(wmesh, oracle.as_blocks(pre[0], pre[1], pre[2].astype(np.float64)),
                                        post, thr, cfg.dt, "xyz", cells=inner)
    assert err <= VAL_TOL * fmax, (err, fmax)
    g.close()


def test_checkpoint_roundtrip_and_restart():
    """Export mid-run, import into a fresh grid, continue: same state as an
    uninterrupted run (restart from a checkpoint, Section 4.2)."""
    n = (20, 12, 9)
    init = inputs.random_blocks(n, (8, 8, 8), 0.3, seed=47)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    a = gpu_grid(mesh, 0.2)
    a.set_blocks(init.off, init.ids, init.vals)
    a.translate(0.2, "xyz", 2, check=True)
    blob = a.export()
    a.translate(0.2, "xyz", 3, check=True)
    b = gpu_grid(mesh, 0.2)
    b.import_(blob)
    b.translate(0.2, "xyz", 3, check=True)
    for x, y in zip(a.get_blocks(), b.get_blocks()):
        np.testing.assert_array_equal(x, y)
    other = gpu_grid(oracle.Mesh(n=(20, 12, 8), nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3), 0.2)
    with pytest.raises(vlasov.VlError) as e:
        other.import_(blob)
    assert e.value.status == vlasov.VL_EINVAL
    with pytest.raises(vlasov.VlError):
        b.import_(blob[:100])


@pytest.mark.parametrize("name, n, origin", [
    ("learned", None, (52, 40, 20)),        # full size: 96x96x48 x 64^3, the rotated rippled front
    ("shock", (128, 64, 32), (56, 9, 5)),   # the shock's structure at half its y extent
])
def test_sparse_config_window_in_captured_steps(name, n, origin):
    """The sparse workloads in the launch configuration the benchmark times (captured
    steps, pools sized by the library): a 16^3 window around the shock front is read
    before and after one step in each form, and the oracle recomputes its 10^3 interior
    from the window (dependence radius 3 per step).  Block sets must match except
    blocks whose oracle maximum is within the guard band of the threshold."""
    import dataclasses
    import torch
    cfg = inputs.CONFIGS[name]
    if n is not None:
        cfg = dataclasses.replace(cfg, n=tuple(n))
    off, ids, vals, thr = inputs.generate_torch(cfg, "cuda")
    size = (16, 16, 16)
    wmesh = oracle.Mesh(n=size, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx, periodic=False)
    inner = [x + size[0] * (y + size[1] * z) for z in range(3, 13) for y in range(3, 13) for x in range(3, 13)]
    posts = []
    for form in ("fused", "3pass"):
        g = gpu_grid(mesh_of(cfg), thr)
        g.set_blocks(off, ids, vals)
        pre = g.get_window(origin, size)
        g.translate(cfg.dt, "xyz", 1, FORMS[form], graph=True, check=True)
        post = g.get_window(origin, size)
        g.close()
        torch.cuda.empty_cache()
        assert pre[1].size > 1000, "the window must hold blocks"
        err, fmax, amb, ref, _ = compare_step(wmesh, oracle.as_blocks(pre[0], pre[1], pre[2].astype(np.float64)),
                                              post, thr, cfg.dt, "xyz", cells=inner)
        assert err <= VAL_TOL * fmax, (form, err, fmax)
        posts.append(post)
    # the two forms agree bit for bit (z-last order)
    for a, b in zip(*posts):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("vmin", [(-3.0, -4.0, -4.5), (-3.0, -2.0, -1.0)])
def test_blocks_straddling_zero_velocity(vmin):
    """Velocity blocks whose cells move both ways along a sweep axis: along x the 3-pass
    form falls back to its one-cell-per-thread kernel (a thread of the vector kernel walks
    four vx cells in one direction); along y and z the threads of a warp walk in
    different directions.  Both forms against the oracle, step by step, and the fused
    form against the 3-pass form (z-last order: bit for bit)."""
    n = (21, 14, 9)
    init = inputs.random_blocks(n, (8, 8, 8), 0.5, seed=48)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=vmin, dv=(1.0,) * 3)
    outs = []
    for form in ("fused", "3pass"):
        g = gpu_grid(mesh, 0.2)
        g.set_blocks(init.off, init.ids, init.vals)
        before = as_ref(init)
        for step in range(2):
            g.translate(0.15, "xyz", 1, FORMS[form], check=True)
            after = g.get_blocks()
            err, fmax, amb, ref, st = compare_step(mesh, before, after, 0.2, 0.15, "xyz")
            assert err <= VAL_TOL * fmax, (form, step, err, fmax)
            before = oracle.as_blocks(*[np.asarray(a) for a in after[:2]], after[2].astype(np.float64))
        outs.append(g.get_blocks())
        g.close()
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("form", ["fused", "3pass"])
def test_mass_and_dropped_mass_with_non_unit_cells(form):
    """Unequal, non-unit cell sizes along every axis (the oracle's volume factor is
    pinned on the same state): every cell holds a block of value 0.75 and one of 0.25;
    with threshold 0.5 and dt = 0 the step drops the second, and the FP64 mass and
    dropped mass equal f times the phase-space volume they cover, which the binary
    fractions make exact."""
    n, dx = (3, 4, 5), (0.5, 1.5, 2.0)
    mesh = oracle.Mesh(n=n, nv=(8, 4, 4), vmin=(-1.0, 0.0, -8.0), dv=(0.25, 0.5, 2.0), dx=dx)
    ncell = int(np.prod(n))
    off = np.arange(ncell + 1, dtype=np.int64) * 2
    ids = np.tile(np.array([0, 1], dtype=np.uint16), ncell)
    vals = np.empty((2 * ncell, 64), dtype=np.float32)
    vals[0::2], vals[1::2] = 0.75, 0.25
    volume = 90.0 * 32.0  # spatial box volume x velocity box volume
    g = gpu_grid(mesh, 0.5)
    g.set_blocks(off, ids, vals)
    assert g.mass() == 0.5 * volume
    assert g.mass() == oracle.mass(mesh, oracle.as_blocks(off, ids, vals.astype(np.float64)))
    g.translate(0.0, "xyz", 1, FORMS[form], check=True)
    s = g.stats()
    assert s.dropped_mass == 0.25 * volume / 2 and s.mass == 0.75 * volume / 2
    assert g.mass() == 0.75 * volume / 2 and g.block_count() == ncell
    g.close()


@pytest.mark.parametrize("storage", [vlasov.VL_STORE_F32, vlasov.VL_STORE_F16_SCALED])
def test_page_locked_host_buffers_are_read_and_written_in_place(storage):
    """vl_set_blocks from page-locked host memory (read in place by the scatter kernel)
    and vl_get_blocks into page-locked host memory (written in place by the gather
    kernel) give the same state as the staged paths from pageable numpy buffers."""
    import torch
    n = (21, 13, 9)
    init = inputs.random_blocks(n, (8, 8, 8), 0.4, seed=95)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    a = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, threshold=0.1, storage=storage)
    a.set_blocks(init.off, init.ids, init.vals)
    a.translate(0.2, "xyz", 1, check=True)
    want = a.get_blocks()
    h_off = torch.from_numpy(init.off.copy()).pin_memory()
    h_ids = torch.from_numpy(init.ids.astype(np.int16)).pin_memory()
    h_vals = torch.from_numpy(init.vals.copy()).pin_memory()
    b = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, threshold=0.1, storage=storage)
    vlasov.vl_set_blocks(b.handle, int(init.ids.size), h_off.data_ptr(), h_ids.data_ptr(), h_vals.data_ptr(), 0)
    b.translate(0.2, "xyz", 1, check=True)
    m = b.block_count()
    o_off = torch.zeros(b.ncells + 1, dtype=torch.int64).pin_memory()
    o_ids = torch.zeros(m, dtype=torch.int16).pin_memory()
    o_vals = torch.full((m, 64), float("nan"), dtype=torch.float32).pin_memory()
    vlasov.vl_get_blocks(b.handle, m, o_off.data_ptr(), o_ids.data_ptr(), o_vals.data_ptr(), 0)
    np.testing.assert_array_equal(o_off.numpy(), want[0])
    np.testing.assert_array_equal(o_ids.numpy().astype(np.uint16), want[1])
    np.testing.assert_array_equal(o_vals.numpy(), want[2])
    a.close()
    b.close()


@pytest.mark.parametrize("n, density, storage", [
    ((1024, 2, 1), 1.0, vlasov.VL_STORE_F32),    # dense: one CTA per pencil group
    ((1024, 2, 1), 0.3, vlasov.VL_STORE_F32),    # sparse: work list, persistent passes
    ((2, 1, 1024), 0.3, vlasov.VL_STORE_F32),    # the longest pencil along z
    ((1024, 1, 2), 0.3, vlasov.VL_STORE_F16_SCALED),
])
def test_longest_pencils(n, density, storage):
    """Pencils of 1024 cells, the longest the 3-pass form holds in shared memory (its rank
    tables and slot bitmaps, one CTA per SM), in both forms against the oracle; a grid
    one cell longer is rejected by the 3-pass form with VL_EINVAL."""
    init = inputs.random_blocks(n, (8, 8, 8), density, seed=49)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    f32 = storage == vlasov.VL_STORE_F32
    # 16-bit storage: no pruning (a block near the threshold may round across it), and
    # the rounding of up to three sweeps (values below 1, so normal float16 codes)
    thr, tol = (0.1, VAL_TOL) if f32 else (0.0, 4 * 2.0 ** -11)
    for form in FORMS.values():
        g = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, threshold=thr, storage=storage)
        g.set_blocks(init.off, init.ids, init.vals)
        off, ids, vals = g.get_blocks()
        before = oracle.as_blocks(off, ids, vals.astype(np.float64))
        g.translate(0.2, "xyz", 1, form, check=True)
        err, fmax, amb, _, _ = compare_step(mesh, before, g.get_blocks(), thr, 0.2, "xyz")
        assert err <= tol * fmax, (form, err, fmax)
        g.close()
    longer = tuple(c + 1 if c == 1024 else c for c in n)
    init = inputs.random_blocks(longer, (8, 8, 8), density, seed=49)
    g = vlasov.Grid(longer, (8, 8, 8), (-4.0,) * 3, (1.0,) * 3, (1.0,) * 3, threshold=thr, storage=storage)
    g.set_blocks(init.off, init.ids, init.vals)
    with pytest.raises(vlasov.VlError) as e:
        g.translate(0.2, "xyz", 1, vlasov.VL_FORM_3PASS, check=True)
    assert e.value.status == vlasov.VL_EINVAL
    g.close()
