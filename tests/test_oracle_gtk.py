"""Pins of the oracle's reduced-ghost (GT1, GT2) tiled step in the form the GPU computes:
tiles along the first two sweep axes, the third axis whole and periodic (box extent 0).

* A second, naive implementation of the region rule of Sections 3.1-3.2, written here
  with plain loops over one tile at a time, must match the oracle to round-off.
* Special cases that make the reduced form exact whatever k: a whole-grid box, and a
  zero Courant number along either tiled axis (that sweep then reads no neighbour, or
  the stale rows equal the swept ones).
* GT3 stays bit-exact; GT1 and GT2 differ from the exact step."""
import numpy as np
import pytest

from naive_ppm import naive_new_value, naive_remap

AX = {"x": 2, "y": 1, "z": 0}  # numpy axis of each physical axis in a [z][y][x] field
H = 3


def naive_gt_step(f, cs, order, k, tile, limiter=True):
    """One GT-k step, tile by tile.  Tile = tile[0] x tile[1] cells along the first two
    sweep axes (ragged at the high end), the third axis whole.  Each tile copies its
    cells plus 3 ghost layers along the two tiled axes from the pre-step field; sweep 0
    updates the tile's cells along axis 0 on the rows within k of the tile along axis 1
    (rows further out keep their copied values), sweep 1 updates the tile's cells, sweep
    2 updates the tile's whole periodic lines; the tile's cells are written back."""
    d0, d1, d2 = order
    f = np.asarray(f, dtype=np.float64)
    # view the field as g[i0][i1][i2] with i_j the coordinate along sweep axis j
    g = np.transpose(f, (AX[d0], AX[d1], AX[d2]))
    n0, n1, n2 = g.shape
    c0, c1, c2 = cs["xyz".index(d0)], cs["xyz".index(d1)], cs["xyz".index(d2)]
    out = g.copy()
    for o0 in range(0, n0, tile[0]):
        for o1 in range(0, n1, tile[1]):
            e0, e1 = min(tile[0], n0 - o0), min(tile[1], n1 - o1)
            # w[u0][u1][i2]: local coordinates u0 - H, u1 - H relative to the tile origin
            w = np.empty((e0 + 2 * H, e1 + 2 * H, n2))
            for u0 in range(e0 + 2 * H):
                for u1 in range(e1 + 2 * H):
                    w[u0, u1, :] = g[(o0 + u0 - H) % n0, (o1 + u1 - H) % n1, :]
            # sweep 0 along axis 0: tile columns, rows -k .. e1+k-1, every plane
            w1 = w.copy()
            for u1 in range(H - k, H + e1 + k):
                for i2 in range(n2):
                    line = list(w[:, u1, i2])
                    for u0 in range(H, H + e0):
                        w1[u0, u1, i2] = naive_new_value(line, u0, c0, limiter)
            # sweep 1 along axis 1: tile cells only
            w2 = w1.copy()
            for u0 in range(H, H + e0):
                for i2 in range(n2):
                    line = list(w1[u0, :, i2])
                    for u1 in range(H, H + e1):
                        w2[u0, u1, i2] = naive_new_value(line, u1, c1, limiter)
            # sweep 2 along the whole periodic axis 2
            for u0 in range(H, H + e0):
                for u1 in range(H, H + e1):
                    out[o0 + u0 - H, o1 + u1 - H, :] = naive_remap(list(w2[u0, u1, :]), c2, limiter)
    inv = np.argsort([AX[d0], AX[d1], AX[d2]])
    return np.transpose(out, inv)


def oracle_box(order, tile):
    """Box extents (x, y, z) of the GPU's tiles for a sweep order: tile[0] along the
    first sweep axis, tile[1] along the second, the third whole (0)."""
    box = [0, 0, 0]
    box["xyz".index(order[0])] = tile[0]
    box["xyz".index(order[1])] = tile[1]
    return tuple(box)


CASES = [
    ((11, 9, 7), "xyz", (4, 3)),   # ragged tiles along both tiled axes
    ((6, 10, 5), "zxy", (3, 4)),
    ((5, 4, 9), "yzx", (2, 4)),    # the ghost layer wraps around the 4-cell axis
]


@pytest.mark.parametrize("n,order,tile", CASES)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_oracle_matches_the_naive_tiled_rule(ref, n, order, tile, k):
    rng = np.random.default_rng(hash((n, order, k)) % 2**32)
    f = rng.uniform(0.0, 1.0, (n[2], n[1], n[0])) ** 2
    cs = [0.83, -0.61, 0.47]
    want = naive_gt_step(f, cs, order, k, tile)
    got = ref.step_field_gt(f, cs, order, True, k, oracle_box(order, tile))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", ["xyz", "zxy"])
def test_whole_axis_boxes_are_exact(ref, order):
    """Boxes spanning every axis have no ghosts at all: every k gives the exact step,
    bit for bit."""
    rng = np.random.default_rng(5)
    f = rng.uniform(0.0, 1.0, (7, 6, 9))
    cs = [0.9, -0.8, 0.35]
    exact = ref.step_field(f, cs, order)
    for k in (1, 2, 3):
        np.testing.assert_array_equal(ref.step_field_gt(f, cs, order, True, k, (0, 0, 0)), exact)


@pytest.mark.parametrize("still", [0, 1])
def test_a_still_tiled_axis_makes_every_k_exact(ref, still):
    """c = 0 along sweep axis 1: that sweep reads no neighbour, so stale rows are never
    used.  c = 0 along sweep axis 0: that sweep changes nothing, so the stale rows hold
    the values the swept ones would.  Either way GT1 = GT2 = GT3 = exact."""
    rng = np.random.default_rng(9 + still)
    f = rng.uniform(0.0, 1.0, (6, 10, 11))
    order = "xyz"
    cs = [0.7, -0.9, 0.6]
    cs[still] = 0.0
    exact = ref.step_field(f, cs, order)
    for k in (1, 2, 3):
        got = ref.step_field_gt(f, cs, order, True, k, oracle_box(order, (4, 3)))
        np.testing.assert_allclose(got, exact, rtol=0, atol=1e-15)


def test_reduced_ghosts_are_approximate_and_gt3_exact(ref):
    rng = np.random.default_rng(13)
    f = rng.uniform(0.0, 1.0, (8, 12, 16))
    cs = [0.8, -0.7, 0.9]
    exact = ref.step_field(f, cs, "xyz")
    box = oracle_box("xyz", (4, 4))
    err = {k: np.abs(ref.step_field_gt(f, cs, "xyz", True, k, box) - exact).max() for k in (1, 2, 3)}
    assert err[3] == 0.0
    assert err[1] > 1e-6 and err[2] > 1e-6
