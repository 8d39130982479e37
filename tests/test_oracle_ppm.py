"""Pins of the oracle's one-dimensional PPM remap against facts fixed by the mathematics
(not by re-typing the oracle's formulas): polynomial exactness, the defining properties of
the limited parabola, the flux as an integral of that parabola, Fourier behaviour of the
linear scheme and convergence against the exact free-streaming solution."""
import math

import numpy as np
import pytest


def cubic_cell_averages(coef, edges):
    """Exact averages of p(x) = sum coef[k] x^k over [edges[i], edges[i+1]]."""
    P = np.polynomial.polynomial.polyint(coef)
    vals = np.polynomial.polynomial.polyval(edges, P)
    return np.diff(vals) / np.diff(edges)


def test_face_value_exact_for_cubics(ref):
    rng = np.random.default_rng(1)
    for _ in range(20):
        coef = rng.normal(size=4)
        x0 = rng.uniform(-3, 3)
        edges = x0 + np.arange(5.0)
        a = cubic_cell_averages(coef, edges)
        f = ref.face(a[0], a[1], a[2], a[3], limiter=False)
        exact = np.polynomial.polynomial.polyval(edges[2], coef)
        assert f == pytest.approx(exact, rel=1e-12, abs=1e-12)


def test_face_clamped_between_neighbours(ref):
    rng = np.random.default_rng(2)
    for _ in range(200):
        a = rng.normal(size=4)
        f = ref.face(*a, limiter=True)
        assert min(a[1], a[2]) <= f <= max(a[1], a[2])
        free = ref.face(*a, limiter=False)
        if min(a[1], a[2]) <= free <= max(a[1], a[2]):
            assert f == free


def parabola_through(aL, a, aR):
    """Coefficients (alpha, beta, gamma) of q(xi) = alpha + beta xi + gamma xi^2 with
    q(0) = aL, q(1) = aR and mean over [0, 1] equal to a (a linear solve)."""
    M = np.array([[1.0, 0.0, 0.0], [1.0, 1.0, 1.0], [1.0, 0.5, 1.0 / 3.0]])
    return np.linalg.solve(M, np.array([aL, aR, a]))


def integrate(coef, lo, hi):
    # 3-point Gauss-Legendre: exact for quadratics, independent of any closed form
    xs, ws = np.polynomial.legendre.leggauss(3)
    t = 0.5 * (hi - lo) * xs + 0.5 * (hi + lo)
    q = coef[0] + coef[1] * t + coef[2] * t * t
    return 0.5 * (hi - lo) * float(np.dot(ws, q))


def test_limited_parabola_is_monotone_and_conservative(ref):
    rng = np.random.default_rng(3)
    for _ in range(2000):
        aL, a, aR = rng.normal(size=3)
        l, r = ref.limit(a, aL, aR)
        if (aR - a) * (a - aL) <= 0:
            assert l == a and r == a  # local extremum: flat cell
            continue
        coef = parabola_through(l, a, r)
        assert integrate(coef, 0.0, 1.0) == pytest.approx(a, rel=1e-12, abs=1e-12)
        d0 = coef[1]
        d1 = coef[1] + 2 * coef[2]
        assert d0 * d1 >= -1e-12 * (1 + abs(d0) + abs(d1)), "parabola has an interior extremum"
        # untouched when the unlimited parabola is already monotone
        c0 = parabola_through(aL, a, aR)
        if c0[1] * (c0[1] + 2 * c0[2]) > 1e-9:
            assert (l, r) == (aL, aR)


def test_outflow_is_integral_of_the_parabola(ref):
    rng = np.random.default_rng(4)
    for _ in range(500):
        aL, a, aR = rng.normal(size=3)
        c = rng.uniform(-1, 1)
        coef = parabola_through(aL, a, aR)
        want = integrate(coef, 1.0 - c, 1.0) if c >= 0 else integrate(coef, 0.0, -c)
        got = ref.outflow(aL, a, aR, c)
        assert got == pytest.approx(want, rel=1e-11, abs=1e-12)
    # the whole cell leaves at |c| = 1, nothing at c = 0
    assert ref.outflow(0.3, 1.7, -2.0, 1.0) == pytest.approx(1.7, rel=1e-15)
    assert ref.outflow(0.3, 1.7, -2.0, -1.0) == pytest.approx(1.7, rel=1e-15)
    assert ref.outflow(0.3, 1.7, -2.0, 0.0) == 0.0


@pytest.mark.parametrize("limiter", [False, True])
def test_quadratic_profiles_advected_exactly(ref, limiter):
    """Averages of a quadratic are remapped to the exact averages of the shifted
    quadratic (reconstruction and flux integral are exact for degree <= 2); with the
    limiter on this holds where the profile is monotone."""
    rng = np.random.default_rng(5)
    n = 40
    edges = np.arange(n + 1.0)
    for _ in range(10):
        coef = np.array([rng.uniform(1, 2), rng.uniform(0.5, 1.0), rng.uniform(0.001, 0.01)])
        if rng.random() < 0.5:
            coef = coef * np.array([1, -1, -1])  # monotone decreasing on [0, 40]
        a = cubic_cell_averages(np.append(coef, 0.0), edges)
        for c in (0.0, 0.3, -0.45, 0.999, -1.0, 1.0):
            out = ref.sweep_line(a, c, limiter=limiter, periodic=False)
            want = cubic_cell_averages(np.append(coef, 0.0), edges - c)
            np.testing.assert_allclose(out[5:-5], want[5:-5], rtol=1e-12, atol=1e-12)


def test_fourier_modes_of_the_linear_scheme(ref):
    n = 64
    x = np.arange(n)
    for k in (1, 3, 7, 15):
        th = 2 * math.pi * k / n
        for c in (0.2, 0.5, -0.7, 1.0, -1.0):
            re = ref.sweep_line(np.cos(th * x), c, limiter=False)
            im = ref.sweep_line(np.sin(th * x), c, limiter=False)
            out = re + 1j * im
            g = out / np.exp(1j * th * x)
            assert np.ptp(g.real) < 1e-12 and np.ptp(g.imag) < 1e-12  # eigenvector
            g = g.mean()
            assert abs(g) <= 1 + 1e-12  # stable for |c| <= 1
            exact = np.exp(-1j * th * c)
            if abs(c) == 1.0:
                assert abs(g - exact) < 1e-12  # whole-cell shift
            else:
                assert abs(g - exact) <= 0.05 * th ** 4 + 1e-13  # third order: O(theta^4)


def l1_error_after(ref, n, c, limiter, t_cells=8.0):
    """Advect f0(x) = 1 + 0.5 sin(2 pi x / L) on n cells over a fixed distance (a
    quarter of the box) and return the L1 error against the exact cell averages."""
    L = float(n)
    steps = int(round(t_cells * n / 32 / c))
    edges = np.arange(n + 1.0)
    a = 1 + 0.5 * (np.cos(2 * np.pi * edges[:-1] / L) - np.cos(2 * np.pi * edges[1:] / L)) * L / (2 * np.pi)
    for _ in range(steps):
        a = ref.sweep_line(a, c, limiter=limiter)
    s = steps * c
    exact = 1 + 0.5 * (np.cos(2 * np.pi * (edges[:-1] - s) / L) - np.cos(2 * np.pi * (edges[1:] - s) / L)) * L / (2 * np.pi)
    return np.abs(a - exact).mean()


def test_convergence_order(ref):
    c = 0.4
    ns = [16, 32, 64, 128]
    for limiter, gate in ((False, 2.8), (True, 1.8)):
        err = [l1_error_after(ref, n, c, limiter) for n in ns]
        orders = [math.log2(err[i] / err[i + 1]) for i in range(len(ns) - 1)]
        assert orders[-1] >= gate, (limiter, err, orders)
