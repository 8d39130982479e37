"""Domain decomposition into z-slabs with one coalesced ghost update per step (Section 3):
the slab bounds, the packing of boundary planes, the routing between neighbours over
torch.distributed (gloo, two and three CPU ranks) and the ghost placement, with the FP64
oracle stepping each rank's local grid.  Every step, the owned planes of every rank equal
the single-domain oracle step bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_2504_21450_gb300 import inputs, slab

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def planes_of(blk, n, z0, nz):
    """Lists of the cells of planes z0 .. z0+nz-1 (wrapping), window order."""
    nxy = n[0] * n[1]
    cells = np.concatenate([np.arange(nxy) + ((z0 + k) % n[2]) * nxy for k in range(nz)])
    cnt = np.diff(blk.off)[cells]
    off = np.zeros(cells.size + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    take = np.concatenate([np.arange(blk.off[c], blk.off[c + 1]) for c in cells]).astype(np.int64)
    return oracle.as_blocks(off, blk.ids[take], blk.vals[take])


def replace_planes(blk, n, z0, nz, new):
    """blk with planes z0 .. z0+nz-1 (wrapping) replaced by the lists `new`."""
    nxy = n[0] * n[1]
    ncell = n[0] * n[1] * n[2]
    src = {}  # cell -> (lists, index of the cell in them)
    for k in range(nz):
        for i in range(nxy):
            src[i + ((z0 + k) % n[2]) * nxy] = k * nxy + i
    off = np.zeros(ncell + 1, dtype=np.int64)
    ids, vals = [], []
    for c in range(ncell):
        if c in src:
            w = src[c]
            a, b = new.off[w], new.off[w + 1]
            ids.append(new.ids[a:b])
            vals.append(new.vals[a:b])
        else:
            a, b = blk.off[c], blk.off[c + 1]
            ids.append(blk.ids[a:b])
            vals.append(blk.vals[a:b])
        off[c + 1] = off[c] + (b - a)
    return oracle.as_blocks(off, np.concatenate(ids), np.concatenate(vals).reshape(-1, 64))


N = (7, 5, 13)
NV = (8, 8, 8)
MESH = dict(nv=NV, vmin=(-4.0, -4.0, -4.0), dv=(1.0, 1.0, 1.0), dx=(1.0, 1.0, 0.8))
THR, DT = 0.2, 0.15


def state():
    init = inputs.random_blocks(N, NV, 0.35, seed=97)
    return oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))


def _rank(rank, world, port, order, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        sl = slab.slabs(N[2], world)[rank]
        gmesh = oracle.Mesh(n=N, **MESH)
        ln = (N[0], N[1], sl.local_nz)
        lmesh = oracle.Mesh(n=ln, **MESH)
        glob = state()
        local = planes_of(glob, N, sl.origin_z, sl.local_nz)
        ex = slab.TorchExchange(sl, dist, "cpu")

        def get(lz0, nz):
            p = planes_of(local, ln, lz0, nz)
            return (torch.from_numpy(p.off), torch.from_numpy(p.ids.astype(np.int16)),
                    torch.from_numpy(p.vals.astype(np.float32)))

        def put(lz0, nz, lists):
            nonlocal local
            off, ids, vals = (t.numpy() for t in lists)
            local = replace_planes(local, ln, lz0, nz,
                                   oracle.as_blocks(off, ids.astype(np.uint16), vals.astype(np.float64)))

        worst = 0
        for _ in range(3):
            # the oracle steps in FP64; the exchange carries float32 values, so both the
            # local and the global state hold float32-representable values at every step
            slab.ghost_update(sl, get, put, ex)
            local = oracle.step(lmesh, local, DT, THR, order)[0]
            glob = oracle.step(gmesh, glob, DT, THR, order)[0]
            local = oracle.as_blocks(local.off, local.ids, local.vals.astype(np.float32).astype(np.float64))
            glob = oracle.as_blocks(glob.off, glob.ids, glob.vals.astype(np.float32).astype(np.float64))
            a = planes_of(local, ln, slab.GHOST, sl.owned)
            b = planes_of(glob, N, sl.z0, sl.owned)
            assert np.array_equal(a.off, b.off) and np.array_equal(a.ids, b.ids)
            worst = max(worst, float(np.abs(a.vals - b.vals).max()) if a.vals.size else 0.0)
        out.put((rank, worst, sl.owned))
    except Exception as e:  # reported to the parent
        out.put((rank, repr(e), -1))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world, order", [(2, "xyz"), (3, "zxy")])
def test_slabs_over_gloo_ranks_equal_the_single_domain_step(world, order):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, order, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (w, n)) for r, w, n in (out.get(timeout=300) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sum(n for _, n in res.values()) == N[2]
    for r in range(world):
        assert res[r][0] == 0.0, res[r]


def test_slab_bounds():
    assert [(s.z0, s.z1) for s in slab.slabs(13, 3)] == [(0, 5), (5, 9), (9, 13)]
    s = slab.slabs(13, 3)[0]
    assert (s.lower, s.upper, s.local_nz, s.origin_z) == (2, 1, 11, -3)
    assert [(t.lower, t.upper) for t in slab.slabs(9, 1)] == [(0, 0)]
    with pytest.raises(ValueError):
        slab.slabs(8, 3)  # a slab of 2 planes cannot hold its neighbours' 3 ghost planes
    sends = [("lo0", "hi0"), ("lo1", "hi1"), ("lo2", "hi2")]
    assert slab.route(slab.slabs(13, 3), sends) == [("hi2", "lo1"), ("hi0", "lo2"), ("hi1", "lo0")]
