"""Pins of the oracle's three-dimensional step: constant states, whole-cell shifts at
|c| = 1, separability and commutation of the split shears, mass conservation and
positivity (Section 2.1 of the paper: three Cartesian shears, mass-conserving remaps,
one face neighbour per step)."""
import numpy as np
import pytest

from paper_2504_21450_gb300 import inputs


def rand_field(shape, seed, lo=0.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


@pytest.mark.parametrize("limiter", [False, True])
def test_constant_state_is_kept(ref, limiter):
    rng = np.random.default_rng(10)
    f = np.full((5, 6, 7), 3.25)
    for _ in range(5):
        c = rng.uniform(-1, 1, size=3)
        out = ref.step_field(f, c, "xyz", limiter)
        np.testing.assert_allclose(out, 3.25, rtol=4e-15)


def test_zero_courant_is_identity(ref):
    f = rand_field((4, 5, 6), 11)
    np.testing.assert_array_equal(ref.step_field(f, [0, 0, 0], "zxy"), f)


def test_whole_cell_shift_at_unit_courant(ref):
    """dx = 1.5, dt = 1, velocity mesh [-2, 2)^3 with dv = 1: the eight corner velocity
    cells have |v_d| = 1.5, i.e. c = +-1 exactly, and must come out as the initial field
    shifted by one cell along (sgn vx, sgn vy, sgn vz)."""
    n = (6, 5, 4)
    mesh = ref.Mesh(n=n, nv=(4, 4, 4), vmin=(-2.0, -2.0, -2.0), dv=(1.0, 1.0, 1.0),
                    dx=(1.5, 1.5, 1.5))
    rng = np.random.default_rng(12)
    ncell = int(np.prod(n))
    blk = ref.as_blocks(np.arange(ncell + 1), np.zeros(ncell), rng.uniform(0.1, 1.0, (ncell, 64)))
    for order in ("xyz", "zxy"):
        out, leaked = ref.translate(mesh, blk, 1.0, order)
        assert leaked == 0.0
        for ivz in (0, 3):
            for ivy in (0, 3):
                for ivx in (0, 3):
                    v = ivx + 4 * (ivy + 4 * ivz)
                    s = (1 if ivx == 3 else -1, 1 if ivy == 3 else -1, 1 if ivz == 3 else -1)
                    f0 = blk.vals[:, v].reshape(n[2], n[1], n[0])
                    want = np.roll(f0, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))
                    got = out.vals[:, v].reshape(n[2], n[1], n[0])
                    np.testing.assert_allclose(got, want, rtol=1e-14)


def test_separable_fields_factor_into_one_dimensional_remaps(ref):
    """The linear (unlimited) step of g(x) h(y) k(z) is (S_x g)(S_y h)(S_z k): each
    shear acts on its own axis only, with its own Courant number."""
    rng = np.random.default_rng(13)
    n = (9, 7, 5)
    g, h, k = (rng.uniform(0, 1, n[d]) for d in range(3))
    f = k[:, None, None] * h[None, :, None] * g[None, None, :]
    c = np.array([0.37, -0.81, 0.55])
    out = ref.step_field(f, c, "yzx", limiter=False)
    sg = ref.sweep_line(g, c[0], limiter=False)
    sh = ref.sweep_line(h, c[1], limiter=False)
    sk = ref.sweep_line(k, c[2], limiter=False)
    want = sk[:, None, None] * sh[None, :, None] * sg[None, None, :]
    np.testing.assert_allclose(out, want, rtol=1e-13, atol=1e-15)


def test_linear_shears_commute(ref):
    f = rand_field((6, 7, 8), 14)
    c = [0.3, -0.6, 0.9]
    a = ref.step_field(f, c, "xyz", limiter=False)
    for order in ("zxy", "yzx", "zyx"):
        np.testing.assert_allclose(ref.step_field(f, c, order, limiter=False), a, rtol=1e-13)


@pytest.mark.parametrize("limiter", [False, True])
def test_mass_is_conserved(ref, limiter):
    rng = np.random.default_rng(15)
    f = rand_field((8, 6, 10), 16)
    for _ in range(3):
        c = rng.uniform(-1, 1, 3)
        out = ref.step_field(f, c, "zxy", limiter)
        assert abs(out.sum() - f.sum()) <= 1e-14 * f.sum()


def test_positivity_with_limiter(ref):
    rng = np.random.default_rng(17)
    f = rand_field((8, 8, 8), 18) ** 4  # sharp, non-negative
    f[f < 0.3] = 0.0
    for _ in range(4):
        c = rng.uniform(-1, 1, 3)
        f = ref.step_field(f, c, "xyz", True)
        assert f.min() >= -1e-15 * f.max()


def test_courant_above_one_is_refused(ref):
    with pytest.raises(ValueError, match="Courant"):
        ref.step_field(np.ones((3, 3, 3)), [1.0000001, 0, 0])


def test_open_box_sees_zero_outside(ref):
    a = np.array([0.0, 0, 0, 1.0, 2.0, 3.0, 0, 0, 0])
    p = ref.sweep_line(a, 0.5, periodic=True)
    o = ref.sweep_line(a, 0.5, periodic=False)
    np.testing.assert_array_equal(p, o)  # zeros around: same as periodic here
    b = np.array([1.0, 2.0, 3.0])
    o = ref.sweep_line(b, 0.5, periodic=False)
    assert o.sum() < b.sum()  # content left through the open right face


def test_maxwellian_moments(ref):
    """n, V and P_dd of a sampled drifting Maxwellian on a fine velocity mesh."""
    cfg = inputs.Config("m", (2, 1, 1), (48, 48, 48), (-12.0, -12.0, -12.0), (0.5, 0.5, 0.5),
                        dt=0.0, steps=0, rel_threshold=0.0, kind="sine",
                        pops=[inputs.Population(1.3, (1.0, -0.5, 0.25), 2.0)])
    init = inputs.generate(cfg)
    mesh = ref.Mesh(n=cfg.n, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv)
    blk = ref.as_blocks(init.off, init.ids, init.vals)
    m = ref.moments(mesh, blk)
    x = np.arange(2) + 0.5
    n_exp = 1.3 * (1 + 0.1 * np.sin(2 * np.pi * x / 2))
    np.testing.assert_allclose(m[:, 0], n_exp, rtol=1e-6)
    np.testing.assert_allclose(m[:, 1:4] / m[:, :1], np.tile([1.0, -0.5, 0.25], (2, 1)), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(m[:, 4:7] / m[:, :1], 4.0, rtol=1e-5)
