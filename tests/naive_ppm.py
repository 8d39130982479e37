"""A deliberately naive PPM remap (Colella & Woodward 1984, eqs. 1.6-1.12) for pins of
the oracle: plain Python loops over explicit indices, no blocks, slots or tiles.  Used
only by tests; it shares nothing with the oracle or the CUDA library."""


def naive_face(a, i, limiter):
    """Value at the face between cells i and i+1 (indices taken modulo len(a)): the
    fourth-order interpolant 7/12 (a_i + a_i+1) - 1/12 (a_i-1 + a_i+2), clamped between
    a_i and a_i+1 when limited."""
    n = len(a)
    v = 7.0 / 12.0 * (a[i % n] + a[(i + 1) % n]) - 1.0 / 12.0 * (a[(i - 1) % n] + a[(i + 2) % n])
    if limiter:
        lo, hi = min(a[i % n], a[(i + 1) % n]), max(a[i % n], a[(i + 1) % n])
        v = min(max(v, lo), hi)
    return v


def naive_parabola(a, i, limiter):
    """(aL, aR) of cell i after CW84's monotonicity constraints (their eq. 1.10)."""
    aL, aR, ai = naive_face(a, i - 1, limiter), naive_face(a, i, limiter), a[i % len(a)]
    if limiter:
        if (aR - ai) * (ai - aL) <= 0.0:
            aL = aR = ai
        else:
            da, mid = aR - aL, 0.5 * (aL + aR)
            if da * (ai - mid) > da * da / 6.0:
                aL = 3.0 * ai - 2.0 * aR
            elif -da * da / 6.0 > da * (ai - mid):
                aR = 3.0 * ai - 2.0 * aL
    return aL, aR


def naive_outflow(a, i, c, limiter):
    """Mass leaving cell i through its downwind face in one remap with Courant number c:
    |c| times the mean of the parabola over the fraction |c| of the cell next to that face
    (CW84 eq. 1.12 with a6 = 6 (a - (aL + aR) / 2))."""
    aL, aR = naive_parabola(a, i, limiter)
    ai = a[i % len(a)]
    da, a6 = aR - aL, 6.0 * (ai - 0.5 * (aL + aR))
    g = abs(c)
    if c >= 0.0:
        return g * (aR - 0.5 * g * (da - (1.0 - 2.0 * g / 3.0) * a6))
    return g * (aL + 0.5 * g * (da + (1.0 - 2.0 * g / 3.0) * a6))


def naive_new_value(a, i, c, limiter):
    """New average of cell i: what does not leave plus the upwind neighbour's outflow.
    Reads cells i-3 .. i+3 of a (modulo len(a))."""
    up = -1 if c >= 0.0 else 1
    return a[i % len(a)] - naive_outflow(a, i, c, limiter) + naive_outflow(a, i + up, c, limiter)


def naive_remap(a, c, limiter):
    """One periodic 1D remap of the whole line."""
    return [naive_new_value(a, i, c, limiter) for i in range(len(a))]
