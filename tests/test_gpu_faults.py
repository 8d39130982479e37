"""Failure detection without a GPU fault: every failure here is made on the host.

* An allocator that stops handing out memory: the call that needed it returns
  VL_ENOMEM, the grid can still be destroyed, and a new grid works.
* The staging-wait timeout path of the fused kernel: with VLGT_FAULT=timeout the kernel
  reports every staging wait that is not complete at its first poll as overdue, then
  waits for it as usual (no copy is left in flight).  The call returns VL_ETIMEOUT, the
  state stays at the last complete step, and the next call works.
Capacity overflow inside captured steps is in test_gpu_graph.py; bad steps, orders and
arguments in test_gpu_parity.py."""
import os

import numpy as np
import pytest

import oracle
from paper_2504_21450_gb300 import inputs, vlasov

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    vlasov.load(build_if_missing=True)


def case():
    n = (24, 10, 9)
    init = inputs.random_blocks(n, (8, 8, 8), 1.0, seed=95)  # dense: bulk staging
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0, -3.0, -4.5), dv=(1.0,) * 3)
    return init, mesh


def run_with_budget(mesh, init, budget):
    """Create, fill and step a grid whose allocator fails after `budget` allocations
    (None: no limit); returns (status of the first failure or None, allocations asked)."""
    import torch
    calls = [0]

    def limited(nbytes):
        calls[0] += 1
        if budget is not None and calls[0] > budget:
            return None
        return int(torch.cuda.caching_allocator_alloc(nbytes))

    g = None
    try:
        g = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, allocator=limited)
        g.set_blocks(init.off, init.ids, init.vals)
        g.translate(0.2, "xyz", 1, check=True)
        failed = None
    except vlasov.VlError as e:
        failed = e.status
    finally:
        if g is not None:
            g.close()
    return failed, calls[0]


def test_allocation_failure_is_reported():
    init, mesh = case()
    failed, total = run_with_budget(mesh, init, None)
    assert failed is None and total > 4
    for budget in (0, 1, total // 2, total - 1):  # creation, set-up, the step
        failed, _ = run_with_budget(mesh, init, budget)
        assert failed == vlasov.VL_ENOMEM, (budget, failed)
    assert run_with_budget(mesh, init, None)[0] is None  # the device is still fine


def test_overdue_staging_wait_is_reported_and_recoverable():
    init, mesh = case()
    ref = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx)
    ref.set_blocks(init.off, init.ids, init.vals)
    ref.translate(0.2, "xyz", 1, vlasov.VL_FORM_FUSED, check=True)
    want = ref.get_blocks()
    ref.close()

    g = vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx)
    g.set_blocks(init.off, init.ids, init.vals)
    os.environ["VLGT_FAULT"] = "timeout"
    try:
        with pytest.raises(vlasov.VlError) as err:
            g.translate(0.2, "xyz", 1, vlasov.VL_FORM_FUSED, check=True)
    finally:
        del os.environ["VLGT_FAULT"]
    assert err.value.status == vlasov.VL_ETIMEOUT
    assert "staging" in str(err.value)
    before = g.get_blocks()  # the failed step did not replace the state
    for a, b in zip(before, (init.off, init.ids, init.vals)):
        np.testing.assert_array_equal(a, b)
    g.translate(0.2, "xyz", 1, vlasov.VL_FORM_FUSED, check=True)  # the context still works
    for a, b in zip(g.get_blocks(), want):
        np.testing.assert_array_equal(a, b)
    g.close()
