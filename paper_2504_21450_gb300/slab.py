"""Spatial domain decomposition into z-slabs with one coalesced ghost update per step.

The paper's Ghost Translation (Section 3) replaces the classical per-direction ghost
updates of Section 2.1 (three per step) by one update of every ghost cell the three sweeps
need, before the step.  Here the spatial domain is split along z over R ranks:

* rank r owns the z-planes [z0_r, z1_r) of the periodic global grid and keeps them in a
  local grid of nz_r + 6 planes: 3 ghost planes below (global z0_r-3 .. z0_r-1), the
  owned planes at local 3 .. nz_r+2, and 3 ghost planes above (global z1_r .. z1_r+2);
* a cell's new value depends only on cells within 3 planes along z (the 2-cell PPM
  stencil plus the face neighbour of the z sweep; the x and y sweeps stay in their plane;
  the block union reaches one plane), so a step of the local grid gives the owned planes
  exactly the values of a step of the global grid.  The local grid is periodic in the
  library's view; its wrap only joins the two ghost layers, whose new values are
  discarded;
* before each step the ghost planes are replaced by the neighbours' boundary planes:
  rank r sends its first 3 owned planes to rank r-1 and its last 3 to rank r+1.

The exchange runs over any transport with ``exchange(send_lo, send_hi) -> (recv_lo,
recv_hi)`` semantics (torch.distributed on GPUs, a loopback for one rank) and any local
engine with ``get_planes`` / ``set_planes`` (the library's vl_get_blocks_window and
vl_set_blocks_planes on the GPU).
"""
from __future__ import annotations

from dataclasses import dataclass

GHOST = 3  # GT3 ghost depth along the decomposed axis


@dataclass(frozen=True)
class Slab:
    rank: int
    world: int
    nz: int      # global planes
    z0: int      # first owned global plane
    z1: int      # one past the last owned plane

    @property
    def owned(self) -> int:
        return self.z1 - self.z0

    @property
    def local_nz(self) -> int:
        return self.owned + 2 * GHOST

    @property
    def origin_z(self) -> int:
        """Global plane of local plane 0 (may be negative: the grid is periodic)."""
        return self.z0 - GHOST

    @property
    def lower(self) -> int:
        """Rank whose last planes are this rank's lower ghosts."""
        return (self.rank - 1) % self.world

    @property
    def upper(self) -> int:
        """Rank whose first planes are this rank's upper ghosts."""
        return (self.rank + 1) % self.world


def slabs(nz: int, world: int) -> list[Slab]:
    """Balanced split of nz planes over `world` ranks (the first nz % world ranks get one
    plane more).  Every slab needs at least GHOST planes: its boundary planes are its
    neighbours' whole ghost layers."""
    if world < 1 or nz < world * GHOST:
        raise ValueError(f"{nz} planes cannot be split over {world} ranks of at least {GHOST} planes")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append(Slab(r, world, nz, z, z + n))
        z += n
    return out


def pack(slab: Slab, get_planes):
    """The boundary planes a rank sends: (first owned planes -> rank `lower`, last owned
    planes -> rank `upper`).  get_planes(lz0, n) returns the per-cell lists of local
    planes lz0 .. lz0+n-1."""
    return get_planes(GHOST, GHOST), get_planes(slab.owned, GHOST)


def unpack(slab: Slab, set_planes, recv_lo, recv_hi) -> None:
    """Replace the ghost planes: recv_lo (the lower rank's last planes) is the lower
    ghost layer (local 0 .. 2), recv_hi (the upper rank's first planes) the upper one
    (local owned+3 .. owned+5).  set_planes(lz0, n, lists) replaces local planes
    lz0 .. lz0+n-1."""
    set_planes(slab.owned + GHOST, GHOST, recv_hi)
    set_planes(0, GHOST, recv_lo)


def route(all_slabs: list[Slab], sends: list):
    """For ranks driven from one process: sends[r] = pack(...) of rank r; returns the
    (recv_lo, recv_hi) of every rank."""
    return [(sends[s.lower][1], sends[s.upper][0]) for s in all_slabs]


def ghost_update(slab: Slab, get_planes, set_planes, exchange) -> None:
    """One coalesced ghost update of a rank's local grid.  exchange(send_lo, send_hi)
    delivers send_lo to rank `lower` and send_hi to rank `upper` and returns (recv_lo,
    recv_hi) = (the lower rank's send_hi, the upper rank's send_lo)."""
    send_lo, send_hi = pack(slab, get_planes)
    recv_lo, recv_hi = exchange(send_lo, send_hi)
    unpack(slab, set_planes, recv_lo, recv_hi)


def loopback(send_lo, send_hi):
    """The exchange of a single rank: its own boundary planes are its ghosts."""
    return send_hi, send_lo


class TorchExchange:
    """Exchange of per-cell lists (off int64 [ncell+1], ids int16 [M], vals float32
    [M][64] tensors) with the two neighbours through torch.distributed point-to-point
    messages.  The lists move in two shifts, first up one rank (send_hi to `upper`,
    recv_lo from `lower`), then down one rank, so that with two ranks, where both
    neighbours are the same peer, each message pair is unambiguous.  Block ids travel as
    bytes (NCCL has no 16-bit integer type)."""

    def __init__(self, slab: Slab, dist, device):
        self.slab = slab
        self.dist = dist
        self.device = device

    def _pair(self, t_send, to: int, like, frm: int):
        dist = self.dist
        buf = like()
        ops = [dist.P2POp(dist.isend, t_send.contiguous(), to), dist.P2POp(dist.irecv, buf, frm)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        return buf

    def _shift(self, lists, to: int, frm: int):
        import torch
        dev = self.device
        off, ids, vals = lists
        m = int(ids.numel())
        cnt = self._pair(torch.tensor([m], dtype=torch.int64, device=dev), to,
                         lambda: torch.zeros(1, dtype=torch.int64, device=dev), frm)
        mr = int(cnt.item())
        off_r = self._pair(off, to, lambda: torch.empty_like(off), frm)
        raw = ids.contiguous().view(torch.uint8) if m else torch.zeros(2, dtype=torch.uint8, device=dev)
        ids_r = self._pair(raw, to, lambda: torch.empty(max(2 * mr, 2), dtype=torch.uint8, device=dev), frm)
        vals_s = vals if m else torch.zeros((1, 64), dtype=torch.float32, device=dev)
        vals_r = self._pair(vals_s, to, lambda: torch.empty((max(mr, 1), 64), dtype=torch.float32, device=dev),
                            frm)
        return off_r, ids_r[: 2 * mr].view(torch.int16), vals_r[:mr]

    def __call__(self, send_lo, send_hi):
        s = self.slab
        if s.world == 1:
            return loopback(send_lo, send_hi)
        recv_lo = self._shift(send_hi, s.upper, s.lower)  # boundary planes move up one rank
        recv_hi = self._shift(send_lo, s.lower, s.upper)  # and down one rank
        return recv_lo, recv_hi


class GridPlanes:
    """get_planes / set_planes of a library grid, with the lists in device tensors."""

    def __init__(self, grid):
        self.g = grid

    def get(self, lz0: int, n: int):
        import torch
        from . import vlasov
        g = self.g
        origin, size = (0, 0, lz0), (g.n[0], g.n[1], n)
        m = vlasov.vl_get_block_count_window(g.handle, origin, size)
        ncell = g.n[0] * g.n[1] * n
        off = torch.empty(ncell + 1, dtype=torch.int64, device=g.device)
        ids = torch.empty(max(m, 1), dtype=torch.int16, device=g.device)
        vals = torch.empty((max(m, 1), 64), dtype=torch.float32, device=g.device)
        vlasov.vl_get_blocks_window(g.handle, origin, size, m, off.data_ptr(), ids.data_ptr(),
                                    vals.data_ptr(), 1)
        return off, ids[:m], vals[:m]

    def set(self, lz0: int, n: int, lists):
        """Local planes lz0 .. lz0+n-1 (wrapping) replaced by the given lists."""
        from . import vlasov
        off, ids, vals = lists
        m = int(ids.numel())
        vlasov.vl_set_blocks_planes(self.g.handle, lz0, n, m, off.data_ptr(),
                                    ids.data_ptr() if m else off.data_ptr(),
                                    vals.data_ptr() if m else off.data_ptr(), 1)
