"""One periodic grid split into z-slabs, one per GPU (rank), with a halo
exchange of g z-layers before every RK stage: the ghost-zone exchange of the
paper's MPI driver (Sec. 2), restated as point-to-point transfers between
neighbouring slabs -- no collective.  On one machine the slabs may also live
in one process (then the exchange is a device copy), which is how the
decomposition is exercised on a single GPU.

Per stage: exchange the z halos of the stage's source state, fill the x and
y ghosts periodically (chemora_fill_ghosts_axes), run the fused stage kernel
(chemora_stage) on every slab.  All arithmetic runs in the library's
kernels; this module only moves ghost layers.

Slab layout: each slab is a grid of nx x ny x n_r points (the same x/y
extent, its own z range [z0, z0 + n_r)) with g ghost layers, padded like any
chemora grid; n_r >= g is required.
"""
import torch

from . import api


def zslabs(nz, nparts):
    """Balanced z ranges: list of (z0, n_r)."""
    if nparts < 1 or nparts > nz:
        raise ValueError("need 1 <= nparts <= nz")
    base, extra = divmod(nz, nparts)
    out, z0 = [], 0
    for r in range(nparts):
        n = base + (1 if r < extra else 0)
        out.append((z0, n))
        z0 += n
    return out


class LocalExchange:
    """Halo exchange between slabs held by this process (a list ordered by
    z)."""

    def __init__(self, g):
        self.g = g

    def __call__(self, states):
        g, P = self.g, len(states)
        lower = [s[:, g:2 * g].clone() for s in states]            # bottom interior layers
        upper = [s[:, -2 * g:-g].clone() for s in states]          # top interior layers
        for r, s in enumerate(states):
            s[:, :g].copy_(upper[(r - 1) % P])
            s[:, -g:].copy_(lower[(r + 1) % P])


class DistExchange:
    """Halo exchange with the neighbouring ranks through torch.distributed
    point-to-point operations (NCCL between GPUs, gloo on CPU).  This rank
    holds one slab; rank r's neighbours are r - 1 and r + 1 modulo the
    world size."""

    def __init__(self, g, rank, world):
        self.g, self.rank, self.world = g, rank, world

    def __call__(self, states):
        import torch.distributed as dist
        (s,) = states
        g, r, P = self.g, self.rank, self.world
        if P == 1:
            LocalExchange(g)(states)
            return
        send_up = s[:, -2 * g:-g].contiguous()   # my top interior -> lower ghosts of r + 1
        send_dn = s[:, g:2 * g].contiguous()     # my bottom interior -> upper ghosts of r - 1
        recv_lo = torch.empty_like(send_up)
        recv_hi = torch.empty_like(send_dn)
        ops = [dist.P2POp(dist.isend, send_up, (r + 1) % P), dist.P2POp(dist.isend, send_dn, (r - 1) % P),
               dist.P2POp(dist.irecv, recv_lo, (r - 1) % P), dist.P2POp(dist.irecv, recv_hi, (r + 1) % P)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        s[:, :g].copy_(recv_lo)
        s[:, -g:].copy_(recv_hi)


class SlabRK4:
    """RK4 on a grid split into z-slabs.  `parts` lists the slabs this
    process owns as (z0, n_r); `exchange` moves the z halos between them."""

    def __init__(self, kind, nx, ny, dx, parts, exchange, params=None, nghost=None):
        self.kind, self.parts, self.exchange = kind, parts, exchange
        self.systems = [api.make_system(kind, nx, ny, n, dx, params=params, nghost=nghost) for _, n in parts]
        self.g = self.systems[0].grid.nghost
        for (_, n) in parts:
            if n < self.g:
                raise ValueError("every slab needs at least %d z-layers" % self.g)
        self.scratch = None

    def _scratch(self, states):
        if self.scratch is None:
            self.scratch = [[torch.zeros_like(s) for _ in range(3)] for s in states]
        return self.scratch

    def fill(self, states):
        """z halos from the neighbours, then periodic x and y ghosts."""
        self.exchange(states)
        for sysm, s in zip(self.systems, states):
            sysm.fill_ghosts_axes(s, 1 | 2)

    def step(self, states, dt, nsteps=1):
        sc = self._scratch(states)
        c2 = (0.5 * dt, 0.5 * dt, dt, 0.0)
        for _ in range(nsteps):
            srcs = [list(states), [x[1] for x in sc], [x[2] for x in sc], [x[1] for x in sc]]
            dsts = [[x[1] for x in sc], [x[2] for x in sc], [x[1] for x in sc], list(states)]
            for q in range(4):
                self.fill(srcs[q])
                for r, sysm in enumerate(self.systems):
                    sysm.stage(q + 1, srcs[q][r], states[r], sc[r][0], dsts[q][r], dt / 6.0, c2[q])
        self.fill(states)
        return states
