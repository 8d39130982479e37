"""Seeded synthetic phase-space inputs (numpy only).

This module is the one piece shared by the oracle side (tests) and the CUDA side
(tests, bench): it builds initial distribution functions and holds none of the
translation method's arithmetic.  The paper's own workloads (a magnetospheric
checkpoint and a flow-through pulse) are not available, so Maxwellian and shock-like
distributions of the same shape stand in for them.

Every distribution is a sum of drifting Maxwellians whose densities vary per
spatial cell:  f(cell, v) = sum_k w_k(cell) * G_k(v),  with
G_k(v) = prod_d exp(-(v_d - V_kd)^2 / (2 vth_k^2)) / (sqrt(2 pi) vth_k)
evaluated at the velocity-cell centres v_d = vmin_d + (i_d + 1/2) dv_d (a point
sample, not a cell average).  Values are rounded to float32, the storage type both
sides start from.

Random perturbations use one splitmix64 round per spatial cell (Steele, Lea & Flood
2014), keyed by the seed and the global cell index, so that any window of a grid gets
exactly the values the full grid has.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(keys: np.ndarray) -> np.ndarray:
    """One splitmix64 output per 64-bit key (wrapping uint64 arithmetic)."""
    z = keys.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, cells: np.ndarray) -> np.ndarray:
    """u in [-1, 1) per global cell index, from splitmix64((seed << 40) ^ cell)."""
    key = (np.uint64(seed) << np.uint64(40)) ^ cells.astype(np.uint64)
    z = splitmix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


@dataclass
class Population:
    n: float
    V: tuple
    vth: float


@dataclass
class Config:
    """One workload: grid, velocity mesh, step and the distribution recipe."""
    name: str
    n: tuple                      # spatial cells (nx, ny, nz), periodic
    nv: tuple                     # velocity cells per dimension
    vmin: tuple
    dv: tuple
    dt: float
    steps: int
    rel_threshold: float          # sparsity threshold relative to the peak of f
    kind: str                     # "sine", "uniform", "shock", "shock_rotated"
    pops: list = field(default_factory=list)
    dx: tuple = (1.0, 1.0, 1.0)
    seed: int = 0
    perturb: float = 0.0          # relative random density perturbation per cell
    front_x: float = 0.0          # shock front position (cells)
    front_width: float = 4.0
    angle_deg: float = 0.0        # front rotation in the x-y plane
    ripple: float = 0.0           # ripple amplitude (cells)
    ripple_wavelength: float = 24.0

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))

    @property
    def nb(self) -> int:
        return int(np.prod([v // 4 for v in self.nv]))


CONFIGS = {
    # plain method, tiny: 8^3 periodic, dense 16^3 velocity mesh on [-8,8)^3
    "tiny": Config("tiny", (8, 8, 8), (16, 16, 16), (-8.0, -8.0, -8.0), (1.0, 1.0, 1.0),
                   dt=0.1, steps=1, rel_threshold=0.0, kind="sine",
                   pops=[Population(1.0, (0.5, 0.0, 0.0), 2.0)]),
    # uniform-mesh scaling: 64^3, 32^3 velocity mesh on [-16,16)^3, 5% density noise
    "uniform": Config("uniform", (64, 64, 64), (32, 32, 32), (-16.0, -16.0, -16.0),
                      (1.0, 1.0, 1.0), dt=0.05, steps=10, rel_threshold=1e-15,
                      kind="uniform", pops=[Population(1.0, (2.0, 1.0, 0.0), 3.0)],
                      perturb=0.05),
    # batched uneven sparsity: tanh shock along x joining a cold beam to a hot sheath
    "shock": Config("shock", (128, 128, 32), (64, 64, 64), (-32.0, -32.0, -32.0),
                    (1.0, 1.0, 1.0), dt=0.025, steps=100, rel_threshold=1e-5, kind="shock",
                    pops=[Population(1.0, (-8.0, 0.0, 0.0), 1.5),
                          Population(0.1, (8.0, 0.0, 0.0), 1.5),
                          Population(4.0, (-2.0, 0.0, 0.0), 6.0)],
                    front_x=64.0),
    # precision form: the uniform distributions on a 32x32x8 periodic grid
    "precision": Config("precision", (32, 32, 8), (32, 32, 32), (-16.0, -16.0, -16.0),
                        (1.0, 1.0, 1.0), dt=0.05, steps=100, rel_threshold=1e-15,
                        kind="uniform", pops=[Population(1.0, (2.0, 1.0, 0.0), 3.0)],
                        perturb=0.05),
    # learned cost model at scale: rotated rippled shock front
    "learned": Config("learned", (96, 96, 48), (64, 64, 64), (-32.0, -32.0, -32.0),
                      (1.0, 1.0, 1.0), dt=0.025, steps=200, rel_threshold=3e-4,
                      kind="shock_rotated",
                      pops=[Population(1.0, (-8.0, 0.0, 0.0), 1.5),
                            Population(0.1, (8.0, 0.0, 0.0), 1.5),
                            Population(4.0, (-2.0, 0.0, 0.0), 6.0)],
                      front_x=48.0, angle_deg=30.0, ripple=3.0),
}


def velocity_centres(nv: int, vmin: float, dv: float) -> np.ndarray:
    return vmin + (np.arange(nv) + 0.5) * dv


def gaussian_1d(v: np.ndarray, V: float, vth: float) -> np.ndarray:
    return np.exp(-((v - V) ** 2) / (2.0 * vth * vth)) / (math.sqrt(2.0 * math.pi) * vth)


def population_tables(cfg: Config) -> np.ndarray:
    """G_k(v) per population as [K, nb, 64] (block id b = bx + nbx*(by + nby*bz),
    value index vx + 4*(vy + 4*vz))."""
    nbx, nby, nbz = (v // 4 for v in cfg.nv)
    out = []
    for p in cfg.pops:
        g = [gaussian_1d(velocity_centres(cfg.nv[d], cfg.vmin[d], cfg.dv[d]), p.V[d], p.vth)
             for d in range(3)]
        G = (g[2][:, None, None] * g[1][None, :, None]) * g[0][None, None, :]  # [vz, vy, vx]
        G = G.reshape(nbz, 4, nby, 4, nbx, 4).transpose(0, 2, 4, 1, 3, 5)
        out.append(G.reshape(nbx * nby * nbz, 64))
    return np.stack(out)


def cell_coords(cfg: Config, cells: np.ndarray):
    nx, ny, _ = cfg.n
    return cells % nx, (cells // nx) % ny, cells // (nx * ny)


def cell_weights(cfg: Config, cells: np.ndarray) -> np.ndarray:
    """Per-cell population densities w_k(cell) as [len(cells), K] (global cell indices)."""
    x, y, z = cell_coords(cfg, cells)
    xc, yc = x + 0.5, y + 0.5
    K = len(cfg.pops)
    w = np.zeros((cells.size, K))
    if cfg.kind == "sine":
        w[:, 0] = cfg.pops[0].n * (1.0 + 0.1 * np.sin(2.0 * math.pi * xc / cfg.n[0]))
    elif cfg.kind == "uniform":
        u = uniform_pm1(cfg.seed, cells)
        w[:, 0] = cfg.pops[0].n * (1.0 + cfg.perturb * u)
    elif cfg.kind in ("shock", "shock_rotated"):
        L = float(cfg.n[0])
        if cfg.kind == "shock":
            # smooth periodic front at x = front_x (mirror front at x = 0), width 4 cells
            s = (L / (2.0 * math.pi * cfg.front_width)) * np.sin(2.0 * math.pi * (xc - cfg.front_x) / L)
        else:
            th = math.radians(cfg.angle_deg)
            xi = (xc - cfg.front_x) * math.cos(th) + (yc - cfg.n[1] / 2.0) * math.sin(th)
            eta = -(xc - cfg.front_x) * math.sin(th) + (yc - cfg.n[1] / 2.0) * math.cos(th)
            phase = 2.0 * math.pi * float(uniform_pm1(cfg.seed, np.array([0]))[0])
            ripple = cfg.ripple * np.sin(2.0 * math.pi * eta / cfg.ripple_wavelength + phase)
            s = (xi - ripple) / cfg.front_width
        up = 0.5 * (1.0 + np.tanh(s))      # upstream (x > front): solar-wind beam
        w[:, 0] = cfg.pops[0].n * up
        w[:, 1] = cfg.pops[1].n * up       # reflected beam, upstream only
        w[:, 2] = cfg.pops[2].n * (1.0 - up)
    else:
        raise ValueError(cfg.kind)
    return w


def peak_f(cfg: Config) -> float:
    """Reference peak of f for the relative threshold: the largest single-population
    peak over the whole grid (exactly max f when there is one population)."""
    G = population_tables(cfg)
    cells = np.arange(cfg.ncells, dtype=np.int64)
    w = cell_weights(cfg, cells)
    return float(max(w[:, k].max() * G[k].max() for k in range(len(cfg.pops))))


def threshold(cfg: Config) -> float:
    return cfg.rel_threshold * peak_f(cfg)


def window_cells(cfg: Config, origin=(0, 0, 0), size=None) -> np.ndarray:
    """Global cell indices of a box window (x fastest), wrapping periodically."""
    size = cfg.n if size is None else size
    x = (origin[0] + np.arange(size[0])) % cfg.n[0]
    y = (origin[1] + np.arange(size[1])) % cfg.n[1]
    z = (origin[2] + np.arange(size[2])) % cfg.n[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return (X + cfg.n[0] * (Y + cfg.n[1] * Z)).reshape(-1).astype(np.int64)


@dataclass
class Initial:
    n: tuple                 # box extents of the generated window
    off: np.ndarray          # int64 [ncells+1]
    ids: np.ndarray          # uint16
    vals: np.ndarray         # float32 [nblocks, 64]
    threshold: float


def generate(cfg: Config, origin=(0, 0, 0), size=None, thr: float | None = None,
             chunk: int = 4096) -> Initial:
    """Initial sparse state of a window: blocks whose float32 maximum reaches the
    threshold are present (all blocks when the threshold is 0)."""
    size = tuple(cfg.n if size is None else size)
    thr = threshold(cfg) if thr is None else thr
    G = population_tables(cfg)
    cells = window_cells(cfg, origin, size)
    offs = [np.zeros(1, dtype=np.int64)]
    ids_l, vals_l = [], []
    total = 0
    for s in range(0, cells.size, chunk):
        cc = cells[s:s + chunk]
        w = cell_weights(cfg, cc)
        f = w[:, 0, None, None] * G[0][None]
        for k in range(1, len(cfg.pops)):
            f = f + w[:, k, None, None] * G[k][None]
        f32 = f.astype(np.float32)
        keep = f32.max(axis=2).astype(np.float64) >= thr
        cnt = keep.sum(axis=1)
        offs.append(total + np.cumsum(cnt))
        total += int(cnt.sum())
        ci, bi = np.nonzero(keep)
        ids_l.append(bi.astype(np.uint16))
        vals_l.append(f32[ci, bi])
    off = np.concatenate(offs).astype(np.int64)
    ids = np.concatenate(ids_l) if ids_l else np.zeros(0, np.uint16)
    vals = np.concatenate(vals_l) if vals_l else np.zeros((0, 64), np.float32)
    return Initial(size, off, ids, np.ascontiguousarray(vals, dtype=np.float32), thr)


def random_blocks(n, nv, density: float, seed: int, scale: float = 1.0,
                  positive: bool = True) -> Initial:
    """Unstructured test state: each (cell, block) present with the given probability,
    values uniform in [0, scale) (or [-scale, scale)), from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    ncell = int(np.prod(n))
    nb = int(np.prod([v // 4 for v in nv]))
    present = rng.random((ncell, nb)) < density
    cnt = present.sum(axis=1)
    off = np.zeros(ncell + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    _, bi = np.nonzero(present)
    v = rng.random((bi.size, 64))
    if not positive:
        v = 2.0 * v - 1.0
    return Initial(tuple(n), off, bi.astype(np.uint16), (scale * v).astype(np.float32), 0.0)


def generate_torch(cfg: Config, device, origin=(0, 0, 0), size=None, thr: float | None = None,
                   chunk: int = 2048):
    """The same initial state as ``generate`` built on a CUDA device with torch (for
    workloads too large for host memory).  The FP64 sum over populations is evaluated in
    the same elementwise order as on the host, so the float32 values agree bit for bit.
    Returns (off, ids, vals, threshold) as CUDA tensors (int64, int32, float32 [M,64])."""
    import torch
    size = tuple(cfg.n if size is None else size)
    thr = threshold(cfg) if thr is None else thr
    G = torch.from_numpy(population_tables(cfg)).to(device)
    cells = window_cells(cfg, origin, size)
    counts = torch.zeros(cells.size, dtype=torch.int64, device=device)
    parts_ids, parts_vals = [], []
    for s in range(0, cells.size, chunk):
        cc = cells[s:s + chunk]
        w = torch.from_numpy(cell_weights(cfg, cc)).to(device)
        f = w[:, 0, None, None] * G[0][None]
        for k in range(1, len(cfg.pops)):
            f = f + w[:, k, None, None] * G[k][None]
        f32 = f.to(torch.float32)
        del f
        keep = f32.amax(dim=2).to(torch.float64) >= thr
        counts[s:s + cc.size] = keep.sum(dim=1)
        ci, bi = torch.nonzero(keep, as_tuple=True)
        parts_ids.append(bi.to(torch.int32))
        parts_vals.append(f32[ci, bi])
        del f32, keep
    off = torch.zeros(cells.size + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=off[1:])
    ids = torch.cat(parts_ids) if parts_ids else torch.zeros(0, dtype=torch.int32, device=device)
    vals = torch.cat(parts_vals) if parts_vals else torch.zeros((0, 64), dtype=torch.float32, device=device)
    return off, ids, vals, thr


def mlp_init(seed: int = 0, nin: int = 8, nh: int = 64) -> np.ndarray:
    """Initial parameters of the cost model's MLP (flat float32, layout W1[nh][nin], b1,
    W2[nh][nh], b2, w3, b3): weights uniform in +-sqrt(6 / (fan_in + fan_out)) (Glorot
    and Bengio 2010), biases 0, from numpy's PCG64 with the given seed."""
    rng = np.random.default_rng(seed)

    def glorot(fan_out, fan_in):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, (fan_out, fan_in))

    parts = [glorot(nh, nin).ravel(), np.zeros(nh), glorot(nh, nh).ravel(), np.zeros(nh),
             glorot(1, nh).ravel(), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)
