"""FP64 oracle of the learned cost model (test infrastructure: only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline may import it; it shares no
code with the CUDA path).

The paper weighs spatial cells by the complexity of their velocity space for load
balancing (Section 2) and points out that the coalesced ghost cells change that cost
(Section 5).  The library predicts the block count of a tile of cells ahead of time with
a small multilayer perceptron; this module states that model plainly:

* tile features (``tile_features``), from the per-cell moments and the block sets;
* regression targets from a trace of union block counts (``targets``);
* y = b3 + w3 . relu(W2 relu(W1 x + b1) + b2) (``forward``), loss (1/n) sum (y - t)^2;
* the gradient by the chain rule (``gradient``) and Adam with bias correction
  (Kingma & Ba 2015, ``adam_step``);
* the pool capacity ceil((1 + margin) sum max(exp(y) - 1, 0)) (``capacity``).

Parameters are one flat vector: W1[64][8] (row = hidden unit), b1[64], W2[64][64],
b2[64], w3[64], b3.
"""
from __future__ import annotations

import numpy as np

import oracle

NIN, NH = 8, 64
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (NPARAM,)
    o = 0
    W1 = p[o:o + NH * NIN].reshape(NH, NIN)
    o += NH * NIN
    b1 = p[o:o + NH]
    o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH)
    o += NH * NH
    b2 = p[o:o + NH]
    o += NH
    w3 = p[o:o + NH]
    o += NH
    return W1, b1, W2, b2, w3, p[o]


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def forward(p, X):
    """y for samples X [n][8], with the layers' pre-activations and outputs."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    return y, (h1, h2)


def loss(p, X, T) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def gradient(p, X, T) -> np.ndarray:
    """dL/dp by the chain rule; the ReLU passes the gradient where its output is > 0."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    y, (h1, h2) = forward(p, X)
    n = X.shape[0]
    dy = 2.0 * (y - np.asarray(T, dtype=np.float64)) / n      # dL/dy        [n]
    da2 = (dy[:, None] * w3[None, :]) * (h2 > 0)                # dL/da2       [n][64]
    da1 = (da2 @ W2) * (h1 > 0)                                 # dL/da1       [n][64]
    return pack(da1.T @ X, da1.sum(axis=0), da2.T @ h1, da2.sum(axis=0), h2.T @ dy, dy.sum())


def adam_step(p, m, v, g, step: int, lr: float):
    """One Adam update (moments m, v; step counts from 1); returns (p, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * g
    v = BETA2 * v + (1.0 - BETA2) * g * g
    mhat = m / (1.0 - BETA1 ** step)
    vhat = v / (1.0 - BETA2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + EPS), m, v


def capacity(p, F, margin: float) -> int:
    y, _ = forward(p, F)
    return int(np.ceil((1.0 + margin) * np.sum(np.maximum(np.expm1(y), 0.0))))


def targets(trace, horizon: int) -> np.ndarray:
    """targets[t][i] = log(1 + max_{0 <= j < horizon} trace[t + j][i])."""
    trace = np.asarray(trace, dtype=np.float64)
    nt = trace.shape[0] - horizon + 1
    return np.log1p(np.stack([trace[t:t + horizon].max(axis=0) for t in range(nt)]))


def tile_ids(n, edge: int) -> np.ndarray:
    """Tile index of every cell (x fastest) for tiles of edge^3 cells, tiles x fastest."""
    nt = [(n[d] + edge - 1) // edge for d in range(3)]
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return ((x // edge) + nt[0] * ((y // edge) + nt[1] * (z // edge))).ravel(), int(np.prod(nt))


def tile_features(mesh: "oracle.Mesh", blk: "oracle.Blocks", edge: int):
    """(features [ntiles][8], union blocks [ntiles]) of a periodic state."""
    n = tuple(mesh.n)
    tid, ntiles = tile_ids(n, edge)
    ncell = int(np.prod(n))
    active = np.diff(blk.off)
    uoff, _ = oracle.union(n, mesh.nb, blk, True)
    uni = np.diff(uoff)
    mom = oracle.moments(mesh, blk)
    nd = mom[:, 0]
    pos = nd > 0
    V = np.zeros((ncell, 3))
    V[pos] = mom[pos, 1:4] / nd[pos, None]
    vth = np.zeros(ncell)
    vth[pos] = np.sqrt(mom[pos, 4:7].sum(axis=1) / (3.0 * nd[pos]))
    ng = nd.reshape(n[2], n[1], n[0])
    g2 = np.zeros_like(ng)
    for ax in range(3):  # array axis 2 is x, 1 is y, 0 is z
        g2 += (0.5 * (np.roll(ng, -1, axis=ax) - np.roll(ng, 1, axis=ax))) ** 2
    grad = np.zeros(ncell)
    grad[pos] = np.sqrt(g2.ravel()[pos]) / nd[pos]
    cnt = np.bincount(tid, minlength=ntiles).astype(np.float64)
    F = np.zeros((ntiles, NIN))
    F[:, 0] = np.log1p(np.bincount(tid, active, ntiles))
    U = np.bincount(tid, uni, ntiles)
    F[:, 1] = np.log1p(U)
    F[:, 2] = np.log1p(np.bincount(tid, nd, ntiles) / cnt)
    for d in range(3):
        F[:, 3 + d] = np.bincount(tid, V[:, d], ntiles) / cnt
    F[:, 6] = np.bincount(tid, vth, ntiles) / cnt
    F[:, 7] = 0.0
    np.maximum.at(F[:, 7], tid, grad)
    return F, U
