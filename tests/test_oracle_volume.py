"""Pins of the oracle's phase-space volume factor and of the density-gradient feature of
the cost model, on states whose answers are known in closed form.

Mass is the integral of f over phase space: with f constant on a box it is f times the
box's spatial volume (n_d dx_d) times its velocity volume (nv_d dv_d), whatever the cell
sizes are (Section 2: the phase-space density f(x, v); the cell sizes only split that
volume into cells).  Every other mass test uses unit cell sizes, where a missing or wrong
volume factor cannot show."""
import numpy as np
import pytest

from oracle import mlp

# a box with unequal, non-unit cell sizes along every axis; velocity blocks do not
# straddle v = 0 (the fused kernel's fast path applies on the GPU)
N = (3, 4, 5)
DX = (0.5, 1.5, 2.0)
NV = (8, 4, 4)
DV = (0.25, 0.5, 2.0)
VMIN = (-1.0, 0.0, -8.0)
SPACE_VOL = 3 * 0.5 * 4 * 1.5 * 5 * 2.0       # 90
VEL_VOL = 8 * 0.25 * 4 * 0.5 * 4 * 2.0        # 32, two blocks of 16


def two_block_state(ref, a, b):
    """Every cell holds block 0 (all values a) and block 1 (all values b)."""
    ncell = int(np.prod(N))
    off = np.arange(ncell + 1, dtype=np.int64) * 2
    ids = np.tile(np.array([0, 1], dtype=np.uint16), ncell)
    vals = np.empty((2 * ncell, 64))
    vals[0::2] = a
    vals[1::2] = b
    return ref.as_blocks(off, ids, vals)


def mesh(ref):
    return ref.Mesh(n=N, nv=NV, vmin=VMIN, dv=DV, dx=DX)


def test_mass_of_a_constant_state_is_f_times_phase_space_volume(ref):
    # 0.75 and the cell sizes are binary fractions: every partial sum is exact
    m = ref.mass(mesh(ref), two_block_state(ref, 0.75, 0.75))
    assert m == 0.75 * SPACE_VOL * VEL_VOL


def test_mass_equals_density_times_spatial_cell_volume(ref):
    """Mass = sum over cells of the density moment n (itself pinned against a sampled
    Maxwellian) times the spatial cell volume."""
    rng = np.random.default_rng(5)
    blk = two_block_state(ref, 0.0, 0.0)
    blk.vals[:] = rng.random(blk.vals.shape)
    me = mesh(ref)
    n = ref.moments(me, blk)[:, 0]
    assert ref.mass(me, blk) == pytest.approx(n.sum() * np.prod(DX), rel=1e-13)


def test_dropped_mass_of_the_sparsity_rule_closed_form(ref):
    """Blocks of value 0.75 stay, blocks of value 0.25 go at threshold 0.5: the dropped
    mass is 0.25 times the phase-space volume the dropped blocks cover (binary fractions
    throughout, so the sums are exact)."""
    me = mesh(ref)
    blk = two_block_state(ref, 0.75, 0.25)
    kept, keep, dropped = ref.prune(me, blk, 0.5)
    np.testing.assert_array_equal(keep, np.tile([1, 0], int(np.prod(N))))
    assert dropped == 0.25 * SPACE_VOL * VEL_VOL / 2
    assert ref.mass(me, kept) == 0.75 * SPACE_VOL * VEL_VOL / 2
    # through a whole step with dt = 0 (nothing moves; the union adds no block)
    after, st, _, _ = ref.step(me, blk, 0.0, 0.5)
    assert st.dropped_mass == 0.25 * SPACE_VOL * VEL_VOL / 2
    assert ref.mass(me, after) == 0.75 * SPACE_VOL * VEL_VOL / 2


def test_density_gradient_feature_of_a_periodic_ramp(ref):
    """n = 1 + 0.1 x on an 8 x 4 x 4 periodic grid (one block of constant f per cell, so
    n = 64 f dv^3): the central difference is 0.1 inside the ramp and -0.3 across the
    periodic step at x = 0 and x = 7, nothing along y and z.  Tiles of 4^3 cells: tile 0
    (x = 0..3) holds max |grad n| / n = 0.3 / 1.0 at x = 0, tile 1 (x = 4..7) holds
    max(0.1/1.4, 0.1/1.5, 0.1/1.6, 0.3/1.7) = 0.3/1.7."""
    n = (8, 4, 4)
    me = ref.Mesh(n=n, nv=(4, 4, 4), vmin=(0.0, 0.0, 0.0), dv=(0.5, 0.5, 0.5))
    ncell = int(np.prod(n))
    x = np.arange(ncell) % n[0]
    dens = 1.0 + 0.1 * x
    off = np.arange(ncell + 1, dtype=np.int64)
    vals = np.repeat((dens / (64 * 0.5 ** 3))[:, None], 64, axis=1)
    blk = ref.as_blocks(off, np.zeros(ncell, dtype=np.uint16), vals)
    np.testing.assert_allclose(ref.moments(me, blk)[:, 0], dens, rtol=1e-14)
    F, _ = mlp.tile_features(me, blk, 4)
    assert F.shape == (2, 8)
    np.testing.assert_allclose(F[:, 7], [0.3, 0.3 / 1.7], rtol=1e-12)
    np.testing.assert_allclose(F[:, 2], np.log1p([1.15, 1.55]), rtol=1e-12)  # mean n per tile
