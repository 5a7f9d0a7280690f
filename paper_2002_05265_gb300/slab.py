"""Single-lattice y-slab decomposition over ranks: host logic only.  Every step of the method
runs in liblbm (lbm_step, lbm_halo_pack, lbm_halo_unpack); this module partitions the rows,
moves the halo messages between ranks and drives the step loop.

One periodic nx x ny lattice (Sec. 5a domains are periodic) is split into `world` slabs of
consecutive rows.  The stream step of Eq. StreamCollide (Sec. 4a) reaches one node, so a slab
only needs, before each step, the populations its neighbours' boundary rows emitted towards it:
the three with xi_y = +1 from the row below and the three with xi_y = -1 from the row above.
A rank's context holds its rows plus one ghost row on each side (local row r = global row
y0 - 1 + r); after every step it packs its boundary rows (send_up, send_down: 3 x nx stored
elements each), exchanges them with the ranks below and above (a periodic ring), and unpacks
what it received into its ghost rows.  The slab's own rows then evolve exactly as the same
rows of the whole lattice (checked bit for bit against one lattice on the GPU and against the
FP64 oracle with gloo ranks on the CPU).
"""

import numpy as np


def slab_rows(ny, rank, world):
    """Rows [y0, y1) of the global lattice owned by `rank`: consecutive, sizes differing by at
    most one, every rank at least one row."""
    if not 1 <= world <= ny:
        raise ValueError(f"cannot split {ny} rows over {world} ranks")
    base, extra = divmod(ny, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def neighbours(rank, world):
    """(rank below, rank above) on the periodic ring of slabs."""
    return (rank - 1) % world, (rank + 1) % world


def local_rows(ny, y0, y1):
    """Global rows held by the local rows 0 .. (y1 - y0) + 1 of a slab (ghosts included)."""
    return np.arange(y0 - 1, y1 + 1) % ny


def exchange(send_up, send_down, recv_below, recv_above, rank, world):
    """Halo exchange of one step: send_up goes to the rank above (its recv_below), send_down to
    the rank below (its recv_above).  One rank: the periodic wrap onto itself.  Several: point
    to point over torch.distributed (NCCL on GPUs, gloo on the CPU), tagged by direction."""
    if world == 1:
        recv_below.copy_(send_up)
        recv_above.copy_(send_down)
        return
    import torch.distributed as dist
    below, above = neighbours(rank, world)
    ops = [dist.P2POp(dist.isend, send_up, above, tag=1), dist.P2POp(dist.irecv, recv_below, below, tag=1),
           dist.P2POp(dist.isend, send_down, below, tag=2), dist.P2POp(dist.irecv, recv_above, above, tag=2)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def advance(n, step_one, pack, unpack, msgs, rank, world):
    """n steps of one rank's slab: step, pack the boundary rows, exchange, unpack into the
    ghost rows.  msgs = (send_up, send_down, recv_below, recv_above)."""
    send_up, send_down, recv_below, recv_above = msgs
    for _ in range(n):
        step_one()
        pack(send_up, send_down)
        exchange(send_up, send_down, recv_below, recv_above, rank, world)
        unpack(recv_below, recv_above)


_RAW = {8: "float64", 4: "float32", 2: "int16"}   # message element type of each storage width


class SlabLattice:
    """One rank's slab of an nx x ny lattice on the GPU: a liblbm context of its rows plus two
    ghost rows, and the four halo message buffers."""

    def __init__(self, nx, ny, model, rates, storage, rank=0, world=1, stream=None, **kw):
        import torch
        from . import lbm
        self.nx, self.ny, self.rank, self.world = nx, ny, rank, world
        self.y0, self.y1 = slab_rows(ny, rank, world)
        self.rows = local_rows(ny, self.y0, self.y1)
        if isinstance(storage, str):
            storage = lbm.STORAGES[storage]
        self.lat = lbm.Lattice(nx, len(self.rows), model, rates, storage=storage, stream=stream, **kw)
        dt = getattr(torch, _RAW[lbm.STORAGE_BYTES[storage]])
        self.msgs = [torch.zeros(3 * nx, dtype=dt, device="cuda") for _ in range(4)]
        self._lbm = lbm

    def close(self):
        self.lat.close()

    def init_equilibrium(self, rho, ux, uy):
        """Global [ny][nx] FP64 fields (torch tensors or numpy arrays); the slab takes its rows
        and the ghost rows from them, so the first step needs no exchange."""
        import torch
        idx = torch.as_tensor(self.rows)
        loc = []
        for a in (rho, ux, uy):
            t = torch.as_tensor(a)
            loc.append(t.index_select(0, idx.to(t.device)).contiguous().to("cuda"))
        self.lat.init_equilibrium(*loc)

    def init_equilibrium_local(self, rho, ux, uy):
        """FP64 fields of the slab's local rows only (global rows `self.rows`, ghosts included),
        [len(rows)][nx] device tensors -- for lattices too large to hold globally per rank."""
        self.lat.init_equilibrium(rho, ux, uy)

    def pack(self, send_up, send_down):
        self._lbm.lbm_halo_pack(self.lat.ctx, send_up, send_down)

    def unpack(self, from_below, from_above):
        self._lbm.lbm_halo_unpack(self.lat.ctx, from_below, from_above)

    def step(self, n):
        advance(n, lambda: self.lat.step(1), self.pack, self.unpack, self.msgs, self.rank, self.world)

    def moments(self, rho=None, ux=None, uy=None):
        """Moments of the slab's own rows ([y1 - y0][nx] FP64 device tensors, any may be None)."""
        import torch
        h = len(self.rows)
        tmp = [torch.empty((h, self.nx), dtype=torch.float64, device="cuda") if o is not None else None
               for o in (rho, ux, uy)]
        self.lat.moments(*tmp)
        for o, t in zip((rho, ux, uy), tmp):
            if o is not None:
                o.copy_(t[1:-1])


def step_slabs(slabs, n):
    """All ranks of a decomposition emulated in one process on one GPU (tests): each step runs
    every slab, packs every slab, then unpacks each slab from its neighbours' messages -- host
    ordered on one stream, no kernel waits on another."""
    world = len(slabs)
    for _ in range(n):
        for s in slabs:
            s.lat.step(1)
            s.pack(s.msgs[0], s.msgs[1])
        for r, s in enumerate(slabs):
            below, above = neighbours(r, world)
            s.unpack(slabs[below].msgs[0], slabs[above].msgs[1])
