"""GT1 and GT2 (reduced ghost depth, Section 3.2) in the fused form against the oracle's
tiled GT-k step with the GPU's tile shape: 16 x TY cells along the first two sweep axes,
the third axis whole and periodic."""
import numpy as np
import pytest

import oracle
from paper_2504_21450_gb300 import inputs, vlasov

from parity import MASS_TOL, VAL_TOL, compare_step, gpu_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    vlasov.load(build_if_missing=True)
    oracle.build()


def box_of(order, ty):
    box = [0, 0, 0]
    box["xyz".index(order[0])] = 16
    box["xyz".index(order[1])] = ty
    return tuple(box)


def case(seed, n=(37, 19, 11)):
    init = inputs.random_blocks(n, (8, 8, 8), 0.3, seed=seed)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0, -3.0, -4.5), dv=(1.0,) * 3)
    return init, mesh, oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))


# (order, tile rows): 16-row tiles with the uniform streamed window, 8-row tiles with
# it, and the sign-generic window of a streamed axis other than z
SHAPES = [("xyz", 16), ("xyz", 8), ("zxy", 8), ("yzx", 8)]


@pytest.mark.parametrize("order,ty", SHAPES)
@pytest.mark.parametrize("k", [1, 2])
def test_reduced_ghost_step_matches_the_oracle(order, ty, k):
    init, mesh, before = case(60 + k)
    thr = 0.05
    g = gpu_grid(mesh, thr)
    g.set_blocks(init.off, init.ids, init.vals)
    g.translate(0.2, order, 1, vlasov.VL_FORM_FUSED, check=True, tile_rows=ty, ghost=k)
    assert g.stats().tile_rows_used == ty
    after = g.get_blocks()
    err, fmax, amb, ref, st = compare_step(mesh, before, after, thr, 0.2, order, gt_k=k,
                                           gt_box=box_of(order, ty))
    assert amb == 0
    assert err <= VAL_TOL * fmax, (err, fmax)
    m_ref = oracle.mass(mesh, ref)
    assert abs(g.mass() - m_ref) <= MASS_TOL * m_ref
    # the reduced form is a different computation: far from the exact step
    exact, _, _, _ = oracle.step(mesh, before, 0.2, thr, order)
    ref_u, _ = oracle.translate(mesh, before, 0.2, order, True, k, box_of(order, ty))
    ex_u, _ = oracle.translate(mesh, before, 0.2, order)
    assert np.abs(ref_u.vals - ex_u.vals).max() > 100 * VAL_TOL * fmax
    g.close()


@pytest.mark.parametrize("k", [1, 2])
def test_reduced_ghost_steps_chain_and_replay_in_a_graph(k):
    """Three steps, as single calls and as one captured graph (whose cache must tell the
    ghost depths apart), against three oracle GT-k steps."""
    init, mesh, before = case(70)
    thr = 0.05
    out = []
    for graph in (False, True):
        g = gpu_grid(mesh, thr)
        g.set_blocks(init.off, init.ids, init.vals)
        if graph:  # a GT3 graph of the same length first: the GT-k call must not replay it
            h = gpu_grid(mesh, thr)
            h.set_blocks(init.off, init.ids, init.vals)
            h.translate(0.2, "xyz", 3, vlasov.VL_FORM_FUSED, check=True, graph=True)
            h.close()
            g.translate(0.2, "xyz", 3, vlasov.VL_FORM_FUSED, check=True, graph=True, ghost=3)
            g.set_blocks(init.off, init.ids, init.vals)
            g.translate(0.2, "xyz", 3, vlasov.VL_FORM_FUSED, check=True, graph=True, ghost=k)
        else:
            for _ in range(3):
                g.translate(0.2, "xyz", 1, vlasov.VL_FORM_FUSED, check=True, ghost=k)
        out.append(g.get_blocks())
        g.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
    blk = before
    for _ in range(3):
        blk, _, _, _ = oracle.step(mesh, blk, 0.2, thr, "xyz", True, k, box_of("xyz", 16))
    err, fmax = 0.0, np.abs(blk.vals).max()
    off, ids, vals = out[0]
    np.testing.assert_array_equal(off, blk.off)
    np.testing.assert_array_equal(ids, blk.ids)
    assert np.abs(vals.astype(np.float64) - blk.vals).max() <= 3 * VAL_TOL * fmax


def test_gt3_is_the_default_and_bit_identical():
    init, mesh, _ = case(71)
    out = []
    for ghost in (None, 3):
        g = gpu_grid(mesh, 0.05)
        g.set_blocks(init.off, init.ids, init.vals)
        if ghost is None:
            g.translate(0.2, "xyz", 2, vlasov.VL_FORM_FUSED, check=True)
        else:
            g.translate(0.2, "xyz", 2, vlasov.VL_FORM_FUSED, check=True, ghost=ghost)
        out.append(g.get_blocks())
        g.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


def test_bad_ghost_requests_are_refused():
    init, mesh, _ = case(72, n=(8, 8, 8))
    g = gpu_grid(mesh, 0.05)
    g.set_blocks(init.off, init.ids, init.vals)
    for form, ghost in ((vlasov.VL_FORM_FUSED, 0), (vlasov.VL_FORM_FUSED, 4),
                        (vlasov.VL_FORM_3PASS, 1), (vlasov.VL_FORM_AUTO, 2)):
        with pytest.raises(vlasov.VlError) as e:
            g.translate(0.2, "xyz", 1, form, check=True, ghost=ghost)
        assert e.value.status == vlasov.VL_EINVAL
    g.close()
    h = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, threshold=0.05,
                    storage=vlasov.VL_STORE_BF16_SCALED)
    h.set_blocks(init.off, init.ids, init.vals)
    with pytest.raises(vlasov.VlError) as e:
        h.translate(0.2, "xyz", 1, vlasov.VL_FORM_FUSED, check=True, ghost=1)
    assert e.value.status == vlasov.VL_EINVAL
    h.close()


def keyed(blocks):
    off, ids, vals = blocks
    cell = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    return cell * 65536 + ids.astype(np.int64), vals.astype(np.float64)


def errors(approx, exact):
    """Relative max and L1 differences of two states over the union of their blocks
    (a block one state lacks counts as zeros)."""
    ka, va = keyed(approx)
    ke, ve = keyed(exact)
    keys = np.union1d(ka, ke)
    A = np.zeros((keys.size, 64))
    E = np.zeros((keys.size, 64))
    A[np.searchsorted(keys, ka)] = va
    E[np.searchsorted(keys, ke)] = ve
    d = np.abs(A - E)
    return d.max() / np.abs(E).max(), d.sum() / np.abs(E).sum()


ERROR_CASES = {
    # the uniform workload's distributions on a 32x32x8 periodic grid, a window of the
    # rotated rippled front (varies along both tiled axes), and a window of the shock,
    # whose profile depends on x only
    "precision": dict(origin=(0, 0, 0), size=None),
    "learned": dict(origin=(16, 32, 0), size=(64, 32, 8)),
    "shock": dict(origin=(32, 0, 0), size=(64, 32, 8)),
}


@pytest.mark.parametrize("name", sorted(ERROR_CASES))
def test_reduced_ghost_error_against_the_exact_step(name):
    """The price of GT1 and GT2 on the workloads' distributions, with the default tile
    (16 x 16), after 1 and 10 steps: relative max and L1 deviation from GT3 (the exact
    step, itself checked against the oracle).  Fewer stale rows, smaller error.  A field
    that does not vary along the second sweep axis (the shock) loses nothing: at the
    stale rows the limiter clamps every face between two equal cells to their value."""
    cfg = inputs.CONFIGS[name]
    init = inputs.generate(cfg, **ERROR_CASES[name])
    out = {}
    for steps in (1, 10):
        res = {}
        for k in (3, 2, 1):
            g = vlasov.Grid(init.n, cfg.nv, cfg.vmin, cfg.dv, cfg.dx, threshold=init.threshold)
            g.set_blocks(init.off, init.ids, init.vals)
            g.translate(cfg.dt, "xyz", steps, vlasov.VL_FORM_FUSED, check=True, ghost=k)
            res[k] = (g.get_blocks(), g.mass())
            g.close()
        for k in (2, 1):
            emax, el1 = errors(res[k][0], res[3][0])
            dm = abs(res[k][1] - res[3][1]) / res[3][1]
            out[(steps, k)] = (emax, el1, dm)
            print(f"{name} steps={steps} GT{k}: rel max {emax:.3e}  rel L1 {el1:.3e}  mass {dm:.3e}")
    for steps in (1, 10):
        if name == "shock":
            assert out[(steps, 1)][0] == 0.0 and out[(steps, 2)][0] == 0.0
        else:
            assert 0.0 < out[(steps, 2)][1] < out[(steps, 1)][1]
            assert out[(steps, 1)][0] < 1.0
