"""Pins of the cost-model oracle (oracle/mlp.py) to things other than itself: central
finite differences for the gradient, hand-built networks with known outputs, Adam's
closed-form first steps, hand-counted tile features of small states."""
import numpy as np
import pytest

import oracle
from oracle import mlp


def rand_params(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, mlp.NPARAM)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = rand_params(2)
    X = rng.normal(0, 1, (12, mlp.NIN))
    T = rng.normal(0, 1, 12)
    g = mlp.gradient(p, X, T)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(mlp.NPARAM):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
    # ReLU kinks are measure-zero for random inputs; central differences are O(h^2)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_forward_of_a_hand_built_network():
    """Hidden unit k (< 8) reads input (k + 3) % 8 with weight k + 1; layer 2 copies
    unit k to unit 7 - k; the output weighs unit j by 10^-j and adds 0.5.  So
    y = 0.5 + sum_k 10^-(7-k) (k + 1) relu(x[(k + 3) % 8])."""
    W1 = np.zeros((64, 8))
    for k in range(8):
        W1[k, (k + 3) % 8] = k + 1
    W2 = np.zeros((64, 64))
    for k in range(8):
        W2[7 - k, k] = 1.0
    w3 = np.zeros(64)
    w3[:8] = 10.0 ** -np.arange(8)
    p = mlp.pack(W1, np.zeros(64), W2, np.zeros(64), w3, 0.5)
    x = np.array([[1.0, -2.0, 3.0, 4.0, -5.0, 6.0, 7.0, 8.0]])
    want = 0.5 + sum(10.0 ** -(7 - k) * (k + 1) * max(x[0, (k + 3) % 8], 0.0) for k in range(8))
    y, _ = mlp.forward(p, x)
    assert y[0] == pytest.approx(want, rel=1e-15)


def test_zero_network_loss():
    T = np.array([1.0, -2.0, 3.0])
    p = np.zeros(mlp.NPARAM)
    p[-1] = 0.25  # b3: the constant output
    assert mlp.loss(p, np.ones((3, 8)), T) == pytest.approx(np.mean((0.25 - T) ** 2))
    g = mlp.gradient(p, np.ones((3, 8)), T)
    assert g[-1] == pytest.approx(2 * np.mean(0.25 - T))
    assert np.all(g[:-1] == 0.0)  # dead ReLUs and zero output weights pass nothing


def test_adam_steps_with_a_constant_gradient():
    """Bias correction makes m_hat = g and v_hat = g^2 at every step for a constant g,
    so each update is -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    for step in (1, 2, 3):
        p, m, v = mlp.adam_step(p, m, v, g, step, 0.01)
        np.testing.assert_allclose(p, -0.01 * step * g / (np.abs(g) + mlp.EPS), rtol=1e-12, atol=1e-18)


def test_targets_and_capacity():
    trace = np.array([[1.0, 5.0], [3.0, 2.0], [0.0, 7.0], [4.0, 1.0]])
    np.testing.assert_allclose(mlp.targets(trace, 2), np.log1p([[3, 5], [3, 7], [4, 7]]))
    p = np.zeros(mlp.NPARAM)
    p[-1] = np.log1p(9.5)  # every tile predicts 9.5 blocks
    assert mlp.capacity(p, np.zeros((4, 8)), 0.1) == int(np.ceil(1.1 * 4 * 9.5))


def test_tile_features_of_a_hand_built_state():
    """One block (id 0, velocity cells all 1/64, so n = 1) in cell (1, 1, 1) of a 6^3
    periodic grid, tiles of 3^3 cells: the block is active in tile 0, and its 27-cell
    union covers cells 0..2 per dimension: all in tile 0."""
    n = (6, 6, 6)
    mesh = oracle.Mesh(n=n, nv=(4, 4, 4), vmin=(-2.0,) * 3, dv=(1.0,) * 3)
    off = np.zeros(217, dtype=np.int64)
    c = 1 + 6 * (1 + 6 * 1)
    off[c + 1:] = 1
    blk = oracle.as_blocks(off, np.array([0], dtype=np.uint16), np.full((1, 64), 1.0 / 64))
    F, U = mlp.tile_features(mesh, blk, 3)
    assert F.shape == (8, 8)
    np.testing.assert_array_equal(U, [27, 0, 0, 0, 0, 0, 0, 0])
    assert F[0, 0] == pytest.approx(np.log(2.0)) and F[0, 1] == pytest.approx(np.log(28.0))
    assert F[0, 2] == pytest.approx(np.log1p(1.0 / 27))  # mean n over the tile's 27 cells
    # the velocity cells are symmetric about 0: V = 0; v_th^2 = mean of v^2 = 1.25
    np.testing.assert_allclose(F[0, 3:6], 0.0, atol=1e-15)
    assert F[0, 6] == pytest.approx(np.sqrt(1.25) / 27)
    # neighbours of (1,1,1) have n = 0: |grad n| = 0 there; at the cell itself the six
    # central differences vanish, so the only non-zero n has zero gradient
    assert F[0, 7] == 0.0
    assert np.all(F[1:, :] == 0.0)
