"""16-bit storage forms (bfloat16 / float16 codes, one power-of-two scale per block id,
FP32 arithmetic): stored values against the IEEE rounding of the oracle's codec, one
step against the FP64 oracle within the rounding bound, invariances (tile rows,
captured graphs, restart from a checkpoint), and the error after several steps of the
32x32x8 precision workload (reported; gated only loosely)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import codec
from paper_2504_21450_gb300 import inputs, vlasov

from parity import VAL_TOL

pytestmark = pytest.mark.gpu

STORES = {"bf16": (vlasov.VL_STORE_BF16_SCALED, codec.BF16),
          "f16": (vlasov.VL_STORE_F16_SCALED, codec.F16)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    vlasov.load(build_if_missing=True)


def grid(mesh, thr, storage):
    return vlasov.Grid(mesh.n, mesh.nv, mesh.vmin, mesh.dv, mesh.dx, threshold=thr, storage=storage)


def wide_case(seed, n=(21, 13, 10)):
    """Random sparse state whose block ids span 27 decades of magnitude (so that float16
    codes need their scales) on an 8^3 velocity mesh."""
    init = inputs.random_blocks(n, (8, 8, 8), 0.4, seed=seed)
    nb = 8
    mag = 10.0 ** np.random.default_rng(seed + 1).uniform(-25, 2, nb)
    vals = (init.vals * mag[init.ids][:, None]).astype(np.float32)
    mesh = oracle.Mesh(n=n, nv=(8, 8, 8), vmin=(-4.0, -3.0, -4.5), dv=(1.0,) * 3)
    return init.off, init.ids, vals, mesh, nb


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_stored_values_are_the_ieee_rounding(name):
    storage, cid = STORES[name]
    off, ids, vals, mesh, nb = wide_case(80)
    g = grid(mesh, 0.0, storage)
    g.set_blocks(off, ids, vals)
    o2, i2, v2 = g.get_blocks()
    np.testing.assert_array_equal(o2, off)
    np.testing.assert_array_equal(i2, ids)
    np.testing.assert_array_equal(v2, codec.encode_decode(ids, vals, nb, cid))
    g.close()


@pytest.mark.parametrize("form", [vlasov.VL_FORM_FUSED, vlasov.VL_FORM_3PASS])
@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_one_step_within_the_rounding_bound(name, form):
    """From the stored state, the FP64 oracle's step and the GPU's differ by the FP32
    arithmetic (the FP32 acceptance tolerance) plus the rounding of the result to the
    storage format: once for the fused form, after each of the three sweeps for the
    3-pass form (bounded there by a few roundings at the block id's scale)."""
    storage, cid = STORES[name]
    off, ids, vals, mesh, nb = wide_case(81)
    g = grid(mesh, 0.0, storage)
    g.set_blocks(off, ids, vals)
    start = g.get_blocks()
    before = oracle.as_blocks(start[0], start[1], start[2].astype(np.float64))
    s_next = codec.block_scales(start[1], start[2], nb)  # the step's output scales
    g.translate(0.2, "xyz", 1, form, check=True)
    o2, i2, v2 = g.get_blocks()
    ref, _, _, _ = oracle.step(mesh, before, 0.2, 0.0, "xyz", True)
    np.testing.assert_array_equal(o2, ref.off)
    np.testing.assert_array_equal(i2, ref.ids)
    err = np.abs(v2.astype(np.float64) - ref.vals)
    s = s_next[ref.ids][:, None].astype(np.float64)
    u = codec.unit_roundoff(cid)
    # the FP32 tolerance is taken per block id (values of one id share a magnitude)
    fmax_id = np.zeros(nb)
    np.maximum.at(fmax_id, ref.ids.astype(np.int64), np.abs(ref.vals).max(axis=1))
    tol32 = VAL_TOL * fmax_id[ref.ids][:, None]
    if form == vlasov.VL_FORM_FUSED:
        bound = u * np.abs(ref.vals) + codec.subnormal_floor(cid) * s + tol32
    else:
        bound = 4 * (u + codec.subnormal_floor(cid)) * s + tol32
    assert np.all(err <= bound), float((err / bound).max())
    g.close()


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_tile_rows_graphs_and_restart_are_bit_identical(name):
    storage, _ = STORES[name]
    off, ids, vals, mesh, nb = wide_case(82)

    def run(nsteps, **kw):
        g = grid(mesh, 1e-3, storage)
        g.set_blocks(off, ids, vals)
        g.translate(0.2, "xyz", nsteps, vlasov.VL_FORM_FUSED, check=True, **kw)
        return g

    a = run(4)
    ref = a.get_blocks()
    for kw in ({"tile_rows": 8}, {"graph": True}):
        b = run(4, **kw)
        for x, y in zip(ref, b.get_blocks()):
            np.testing.assert_array_equal(x, y)
        b.close()
    c = run(2)
    blob = c.export()
    c.close()
    d = grid(mesh, 1e-3, storage)
    d.import_(blob)
    d.translate(0.2, "xyz", 2, vlasov.VL_FORM_FUSED, check=True)
    for x, y in zip(ref, d.get_blocks()):
        np.testing.assert_array_equal(x, y)
    other = grid(mesh, 1e-3, vlasov.VL_STORE_F32)
    with pytest.raises(vlasov.VlError):
        other.import_(blob)  # storage type differs
    for h in (a, d, other):
        h.close()


def test_auto_form_with_16bit_storage_tunes_tiles_only():
    off, ids, vals, mesh, nb = wide_case(83)
    g = grid(mesh, 0.0, vlasov.VL_STORE_BF16_SCALED)
    g.set_blocks(off, ids, vals)
    g.translate(0.2, "xyz", 6, vlasov.VL_FORM_AUTO, check=True)
    s = g.stats()
    assert s.form_used == vlasov.VL_FORM_FUSED and s.tune_ms[3] == 0.0
    g.close()


def test_precision_workload_error_report():
    """The 32x32x8 periodic grid with the uniform workload's distributions (32^3
    velocity cells, 5% density noise): 10 steps (VLGT_PRECISION_STEPS to change) in FP32,
    bfloat16 and float16 storage against the FP64 oracle from the same float32 input.
    FP32 meets the acceptance tolerance; the 16-bit errors are reported (max-abs, L1 and
    L2 relative to the oracle's max, L1 and L2 norms, and the mass change) and gated only
    at a few units of their rounding."""
    cfg = inputs.CONFIGS["precision"]
    nsteps = int(os.environ.get("VLGT_PRECISION_STEPS", "10"))
    init = inputs.generate(cfg)
    off, ids, vals, thr = init.off, init.ids, init.vals, init.threshold
    mesh = oracle.Mesh(n=cfg.n, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx)
    ref = oracle.as_blocks(off, ids, vals.astype(np.float64))
    m0 = oracle.mass(mesh, ref)
    for _ in range(nsteps):
        ref, _, _, _ = oracle.step(mesh, ref, cfg.dt, thr, "xyz", True)
    rk = ref.off
    fmax = float(np.abs(ref.vals).max())
    report = {"workload": f"precision: {cfg.n} cells x {cfg.nv} velocity cells, {nsteps} steps",
              "fmax": fmax}
    for name, storage in (("f32", vlasov.VL_STORE_F32), ("bf16", vlasov.VL_STORE_BF16_SCALED),
                          ("f16", vlasov.VL_STORE_F16_SCALED)):
        for form, fname in ((vlasov.VL_FORM_FUSED, "fused"), (vlasov.VL_FORM_3PASS, "3pass")):
            g = grid(mesh, thr, storage)
            g.set_blocks(off, ids, vals)
            g.translate(cfg.dt, "xyz", nsteps, form, check=True)
            o2, i2, v2 = g.get_blocks()
            mass = g.mass()
            g.close()
            same = np.array_equal(o2, rk) and np.array_equal(i2, ref.ids)
            entry = {"same_block_set": bool(same), "mass_change": (mass - m0) / m0}
            if same:
                d = np.abs(v2.astype(np.float64) - ref.vals)
                entry["max_abs_rel"] = float(d.max()) / fmax
                entry["l1_rel"] = float(d.sum() / np.abs(ref.vals).sum())
                entry["l2_rel"] = float(np.sqrt((d * d).sum() / (ref.vals * ref.vals).sum()))
            report[f"{name}_{fname}"] = entry
    print(json.dumps(report))
    path = os.environ.get("VLGT_PRECISION_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(report, fh, indent=1)
    for fname in ("fused", "3pass"):
        assert report[f"f32_{fname}"]["same_block_set"]
        assert report[f"f32_{fname}"]["max_abs_rel"] <= VAL_TOL
        for name, cid in (("bf16", codec.BF16), ("f16", codec.F16)):
            e = report[f"{name}_{fname}"]
            if e["same_block_set"]:
                assert e["max_abs_rel"] <= 4 * nsteps * codec.unit_roundoff(cid)
