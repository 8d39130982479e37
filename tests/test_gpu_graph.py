"""Captured step sequences (CUDA graphs): no host synchronisation between steps, pools
pre-sized to a capacity with device-side overflow detection and recovery.  The state
must be bit-identical to step-by-step execution."""
import numpy as np
import pytest

import oracle
from paper_2504_21450_gb300 import inputs, vlasov

from parity import VAL_TOL, compare_step, gpu_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    vlasov.load(build_if_missing=True)


def sparse_case(seed):
    n = (33, 17, 20)
    init = inputs.random_blocks(n, (8, 8, 8), 0.15, seed=seed)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0, -3.0, -4.5), dv=(1.0,) * 3)
    return init, mesh


def run(mesh, init, thr, nsteps, form, graph, capacity=0, calls=1):
    g = gpu_grid(mesh, thr)
    g.set_blocks(init.off, init.ids, init.vals)
    stats = []
    for _ in range(calls):
        g.translate(0.2, "xyz", nsteps, form, graph=graph, capacity=capacity, check=True)
        stats.append(g.stats())
    out = g.get_blocks()
    g.close()
    return out, stats


@pytest.mark.parametrize("form", [vlasov.VL_FORM_FUSED, vlasov.VL_FORM_3PASS])
def test_graph_equals_step_by_step(form):
    init, mesh = sparse_case(60)
    ref, rs = run(mesh, init, 0.2, 6, form, graph=False)
    got, gs = run(mesh, init, 0.2, 6, form, graph=True)
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    assert gs[0].steps == 6 and gs[0].graph_replays == 1 + gs[0].capacity_regrows
    assert gs[0].blocks == rs[0].blocks and gs[0].dropped_blocks == rs[0].dropped_blocks
    assert abs(gs[0].mass - rs[0].mass) <= 1e-12 * rs[0].mass
    assert gs[0].launches > 0


def test_capacity_overflow_is_recovered():
    """Pools sized below what the growing block union needs: the overflowing step is
    detected on the device, the state stays at the last complete step, the pools grow
    and the remaining steps run again -- with the same result."""
    init, mesh = sparse_case(61)
    ref, _ = run(mesh, init, 0.0, 5, vlasov.VL_FORM_FUSED, graph=False)
    got, gs = run(mesh, init, 0.0, 5, vlasov.VL_FORM_FUSED, graph=True, capacity=int(init.off[-1]))
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    assert gs[0].capacity_regrows >= 1 and gs[0].graph_replays >= 2
    assert gs[0].capacity > init.off[-1]


def test_cached_graph_is_replayed():
    init, mesh = sparse_case(62)
    ref, _ = run(mesh, init, 0.0, 8, vlasov.VL_FORM_FUSED, graph=False)
    full = mesh.ncells * mesh.nb  # every (cell, block id) pair: no overflow possible
    got, gs = run(mesh, init, 0.0, 4, vlasov.VL_FORM_FUSED, graph=True, capacity=full, calls=2)
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    assert [s.graph_replays for s in gs] == [1, 1] and [s.steps for s in gs] == [4, 4]


def test_graph_steps_match_oracle():
    init, mesh = sparse_case(63)
    g = gpu_grid(mesh, 0.3)
    g.set_blocks(init.off, init.ids, init.vals)
    before = oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))
    for _ in range(2):
        g.translate(0.2, "xyz", 1, vlasov.VL_FORM_FUSED, graph=True, check=True)
        after = g.get_blocks()
        err, fmax, _, _, _ = compare_step(mesh, before, after, 0.3, 0.2, "xyz")
        assert err <= VAL_TOL * fmax
        before = oracle.as_blocks(after[0], after[1], after[2].astype(np.float64))
