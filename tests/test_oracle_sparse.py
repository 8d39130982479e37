"""Pins of the oracle's sparse velocity space (Section 2: 64-element blocks added where
a neighbour can send content and removed below the sparsity threshold)."""
import numpy as np
import pytest

from paper_2504_21450_gb300 import inputs


def presence(n, nb, off, ids):
    ncell = int(np.prod(n))
    P = np.zeros((ncell, nb), dtype=bool)
    cell = np.repeat(np.arange(ncell), np.diff(off))
    P[cell, ids] = True
    return P.reshape(n[2], n[1], n[0], nb)


def test_union_is_the_27_cell_dilation(ref):
    n, nv = (5, 4, 6), (8, 8, 4)
    init = inputs.random_blocks(n, nv, 0.05, seed=30)
    blk = ref.as_blocks(init.off, init.ids, init.vals)
    nb = 2 * 2 * 1
    off_u, ids_u = ref.union(n, nb, blk)
    P = presence(n, nb, init.off, init.ids)
    D = np.zeros_like(P)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                D |= np.roll(P, (dz, dy, dx), axis=(0, 1, 2))
    np.testing.assert_array_equal(presence(n, nb, off_u, ids_u), D)
    # ids sorted per cell
    for c in range(int(np.prod(n))):
        s = ids_u[off_u[c]:off_u[c + 1]]
        assert np.all(np.diff(s.astype(int)) > 0)


def test_open_box_union_stays_inside(ref):
    n = (3, 3, 3)
    off = np.zeros(28, dtype=np.int64)
    off[1:] = 0
    off[14:] = 1  # one block in the centre cell (index 13)
    blk = ref.as_blocks(off, np.array([0], dtype=np.uint16), np.ones((1, 64)))
    off_u, ids_u = ref.union(n, 1, blk, periodic=False)
    assert off_u[-1] == 27
    off2 = np.zeros(28, dtype=np.int64)
    off2[1:] = 1  # one block in corner cell 0
    blk2 = ref.as_blocks(off2, np.array([0], dtype=np.uint16), np.ones((1, 64)))
    assert ref.union(n, 1, blk2, periodic=False)[0][-1] == 8
    assert ref.union(n, 1, blk2, periodic=True)[0][-1] == 27


def test_nothing_leaks_outside_the_union(ref):
    init = inputs.random_blocks((6, 5, 7), (8, 8, 8), 0.1, seed=31)
    mesh = ref.Mesh(n=(6, 5, 7), nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    blk = ref.as_blocks(init.off, init.ids, init.vals)
    for order in ("xyz", "zyx"):
        u, leaked = ref.translate(mesh, blk, 0.25, order)
        assert leaked == 0.0


def test_mass_conserved_up_to_dropped_mass(ref):
    init = inputs.random_blocks((6, 6, 6), (8, 8, 8), 0.2, seed=32)
    mesh = ref.Mesh(n=(6, 6, 6), nv=(8, 8, 8), vmin=(-4.0,) * 3, dv=(1.0,) * 3)
    blk = ref.as_blocks(init.off, init.ids, init.vals * (np.arange(init.ids.size) % 7 == 0)[:, None] + 1e-9 * init.vals)
    m0 = ref.mass(mesh, blk)
    thr = 1e-3
    kept, st, u, keep = ref.step(mesh, blk, 0.2, thr)
    assert st.leaked == 0.0
    assert 0 < st.kept_blocks < st.union_blocks
    assert st.dropped_mass > 0
    assert abs(ref.mass(mesh, kept) + st.dropped_mass - m0) <= 1e-13 * m0
    # threshold 0 keeps every union block and conserves mass to round-off
    kept0, st0, _, _ = ref.step(mesh, blk, 0.2, 0.0)
    assert st0.kept_blocks == st0.union_blocks and st0.dropped_mass == 0.0
    assert abs(ref.mass(mesh, kept0) - m0) <= 1e-14 * m0


def test_prune_keeps_ties(ref):
    mesh = ref.Mesh(n=(2, 1, 1), nv=(4, 4, 4), vmin=(-2.0,) * 3, dv=(1.0,) * 3)
    v = np.zeros((2, 64))
    v[0, 5] = 0.5
    v[1, 7] = 0.4999999
    blk = ref.as_blocks([0, 1, 2], [0, 0], v)
    kept, keep, dropped = ref.prune(mesh, blk, 0.5)
    assert list(keep) == [1, 0]
    assert dropped == pytest.approx(0.4999999)
    assert list(kept.off) == [0, 1, 1]


def test_block_machinery_matches_dense_fields(ref):
    """Brute force on a 4x4x4 grid holding one dense 4x4x4 velocity block: the sparse
    step equals advancing each of the 64 velocity cells as a plain dense field with its
    own Courant numbers (v-cell index vx + 4 vy + 16 vz, centres at vmin + (i + 1/2) dv)."""
    n = (4, 4, 4)
    mesh = ref.Mesh(n=n, nv=(4, 4, 4), vmin=(-2.0, -1.0, -3.0), dv=(1.0, 0.5, 1.5), dx=(1.0, 2.0, 1.5))
    rng = np.random.default_rng(33)
    vals = rng.uniform(0, 1, (64, 64))
    blk = ref.as_blocks(np.arange(65), np.zeros(64), vals)
    dt = 0.4
    for order in ("xyz", "yzx"):
        u, _ = ref.translate(mesh, blk, dt, order)
        for v in range(64):
            iv = (v % 4, (v // 4) % 4, v // 16)
            c = [(mesh.vmin[d] + (iv[d] + 0.5) * mesh.dv[d]) * dt / mesh.dx[d] for d in range(3)]
            f = vals[:, v].reshape(4, 4, 4)
            want = ref.step_field(f, c, order)
            np.testing.assert_array_equal(u.vals[:, v].reshape(4, 4, 4), want)


def test_generator_windows_match_full_grid():
    cfg = inputs.CONFIGS["uniform"]
    small = inputs.Config(**{**cfg.__dict__, "n": (8, 8, 8), "nv": (8, 8, 8), "vmin": (-4.0,) * 3})
    full = inputs.generate(small, thr=0.0)
    win = inputs.generate(small, origin=(6, 2, 7), size=(4, 3, 2), thr=0.0)
    cells = inputs.window_cells(small, (6, 2, 7), (4, 3, 2))
    for i, c in enumerate(cells):
        a = full.vals[full.off[c]:full.off[c + 1]]
        b = win.vals[win.off[i]:win.off[i + 1]]
        np.testing.assert_array_equal(a, b)


def test_configs_have_the_stated_shape():
    tiny = inputs.generate(inputs.CONFIGS["tiny"])
    assert tiny.n == (8, 8, 8) and tiny.off[-1] == 512 * 64  # dense 16^3 mesh
    cfg = inputs.CONFIGS["uniform"]
    w = inputs.generate(cfg, size=(2, 2, 2))
    assert w.off[-1] == 8 * 512  # 1e-15 of the peak keeps every block
    u = inputs.uniform_pm1(0, np.arange(100000))
    assert -1 <= u.min() < -0.99 and 0.99 < u.max() < 1 and abs(u.mean()) < 0.01
