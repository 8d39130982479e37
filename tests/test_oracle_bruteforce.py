"""Brute force on a 4x4x4 periodic grid holding one dense 4x4x4 velocity block, against a
second, deliberately naive implementation written here from Colella & Woodward (1984):
plain Python loops with explicit modular indexing, no blocks, no slots, no tiles.

* Limited scheme: every one of the 64 velocity cells (Courant numbers of both signs, up
  to |c| = 1) matches the oracle's sparse step to round-off.
* Linear scheme (limiter off): the oracle's step, applied to the 64 unit fields, is a
  64x64 matrix that equals the Kronecker product of three 4x4 circulant matrices built
  from the naive 1D remap -- one per sweep axis, the shears commuting.
A halo of 3 cells on a 4-cell periodic line wraps onto the line itself, which makes this
grid an edge case for any ghost-cell indexing."""
import numpy as np
import pytest

import oracle
from naive_ppm import naive_remap


def naive_step(field, cs, order, limiter):
    """x->y->z (or any order) shears of a [z][y][x] field, each line remapped naively."""
    f = np.array(field, dtype=np.float64)
    axis_of = {"x": 2, "y": 1, "z": 0}
    for d in order:
        ax = axis_of[d]
        c = cs["xyz".index(d)]
        g = np.moveaxis(f, ax, -1).copy()
        for idx in np.ndindex(g.shape[:-1]):
            g[idx] = naive_remap(list(g[idx]), c, limiter)
        f = np.moveaxis(g, -1, ax)
    return f


def courants(mesh, dt):
    """Courant number of every velocity cell v = vx + 4 vy + 16 vz of the one block."""
    out = []
    for v in range(64):
        iv = (v % 4, (v // 4) % 4, v // 16)
        out.append([(mesh.vmin[d] + (iv[d] + 0.5) * mesh.dv[d]) * dt / mesh.dx[d] for d in range(3)])
    return out


# velocity mesh chosen so that along every axis the 4 cells move both ways and the
# largest |c| is exactly 1 (dt = 1, dx = 1.5: v = -1.5, -0.5, 0.5, 1.5 -> c = -1, ..., 1)
MESH = dict(n=(4, 4, 4), nv=(4, 4, 4), vmin=(-2.0, -2.0, -2.0), dv=(1.0, 1.0, 1.0), dx=(1.5, 1.5, 1.5))


@pytest.mark.parametrize("order", ["xyz", "zxy"])
def test_limited_step_matches_the_naive_remap_for_all_64_velocity_cells(order):
    mesh = oracle.Mesh(**MESH)
    dt = 1.0
    rng = np.random.default_rng(51)
    vals = rng.uniform(0.0, 1.0, (64, 64))  # [cell][velocity cell]
    blk = oracle.as_blocks(np.arange(65), np.zeros(64), vals)
    got, leaked = oracle.translate(mesh, blk, dt, order, limiter=True)
    assert leaked == 0.0
    np.testing.assert_array_equal(got.off, np.arange(65))
    cs = courants(mesh, dt)
    assert {abs(c[0]) for c in cs} == {1.0 / 3.0, 1.0} and min(c[0] for c in cs) < 0 < max(c[0] for c in cs)
    for v in range(64):
        f = vals[:, v].reshape(4, 4, 4)  # cell index x + 4 y + 16 z -> [z][y][x]
        want = naive_step(f, cs[v], order, True)
        np.testing.assert_allclose(got.vals[:, v].reshape(4, 4, 4), want, rtol=0, atol=1e-14)


def test_linear_step_is_a_kronecker_product_of_circulants():
    mesh = oracle.Mesh(**dict(MESH, dx=(3.0, 2.5, 1.75)))  # |c| below 1, different per axis
    dt = 0.7
    cs = courants(mesh, dt)
    # the oracle's step on the 64 unit fields of every velocity cell at once: column j of
    # the operator of velocity cell v is the step of the unit field of cell j
    for v in (0, 21, 42, 63):  # corners and interior velocity cells, signs differ
        vals = np.zeros((64, 64))
        M = np.zeros((64, 64))
        for j in range(64):
            vals[:] = 0.0
            vals[j, v] = 1.0
            blk = oracle.as_blocks(np.arange(65), np.zeros(64), vals)
            got, _ = oracle.translate(mesh, blk, dt, "xyz", limiter=False)
            M[:, j] = got.vals[:, v]
        # 1D operators from the naive remap, as 4x4 matrices (columns = unit inputs)
        ops = []
        for d in range(3):
            A = np.array([naive_remap(list(np.eye(4)[j]), cs[v][d], False) for j in range(4)]).T
            for s in range(4):  # circulant: invariant under cyclic shifts
                np.testing.assert_allclose(np.roll(np.roll(A, s, 0), s, 1), A, atol=1e-15)
            np.testing.assert_allclose(A.sum(axis=0), 1.0, atol=1e-15)  # conserves mass
            ops.append(A)
        # cell index x + 4 y + 16 z: z is the slowest index, so M = Az (x) Ay (x) Ax
        K = np.kron(ops[2], np.kron(ops[1], ops[0]))
        np.testing.assert_allclose(M, K, rtol=0, atol=1e-14)
