"""Particles sharded over processes (one GPU each) and the one exchange step
of the particle path.

Particles do not interact within a step: each process holds the whole mesh
and envelope DoFs and advances its own range of particles, and the only
coupling is the step's edge deposit dG (Sec. III-D eq. G_integral), summed
over the shards.  A rank finalizes its own dG (fempic_deposit_local), the
ranks all-reduce it, and each adds the sum to its cumulative G
(fempic_accumulate), so G_cum and the envelope-frame G~ are the same on every
rank and equal to an unsharded run's up to summation order.  The adjoint's
DoF gradients are summed the same way; per-particle gradients stay with
their rank.

The shards are contiguous ranges of the tet-sorted particle set, so each
rank's particles start in one block of tets: the same per-tet locality as
one process holds.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from .env import FempicEnv, ParticleState
from .inputs import Particles


def allreduce_(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum over the group's ranks; device tensors go through host
    copies when the backend cannot reduce device memory (gloo)."""
    if dist.get_backend(group) == "gloo" and t.is_cuda:
        h = t.cpu()
        dist.all_reduce(h, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, group=group)
    return t


def tet_range(st_sorted: ParticleState, rank: int, world: int) -> ParticleState:
    """Rank's contiguous range of a particle set already sorted by
    (species, tet): equal particle counts per rank, species table restricted
    to the range.  The arrays are copies."""
    n = st_sorted.n
    a, b = rank * n // world, (rank + 1) * n // world
    sb = np.clip(st_sorted.species_begin - a, 0, b - a).astype(np.int64)
    c = lambda t: None if t is None else t[a:b].clone()
    out = ParticleState(c(st_sorted.x), c(st_sorted.y), c(st_sorted.z), c(st_sorted.vx), c(st_sorted.vy),
                        c(st_sorted.vz), sb, st_sorted.q, st_sorted.m, st_sorted.w, tet=c(st_sorted.tet),
                        track_crossings=st_sorted.n_cross is not None)
    out.status = c(st_sorted.status)
    if st_sorted.n_cross is not None:
        out.n_cross = c(st_sorted.n_cross)
    return out


def slab_load(parts: Particles, rank: int, world: int, axis: int = 2, lo: float = 0.0, hi: float = 1.0) -> Particles:
    """Rank's share of a load that is uniform along `axis` over [lo, hi]: the
    rank's own draw with that coordinate mapped into slab `rank` of `world`
    equal slabs.  The union over ranks is a uniform load of world times the
    particles, and each rank's share is the slab's particles; on a Kuhn cube
    whose cell count along z is a multiple of world, a z-slab is a
    contiguous range of tet ids, so this is the tet-range partition of that
    global load, without drawing the global load on every rank."""
    if world == 1:
        return parts
    cols = [parts.x.copy(), parts.y.copy(), parts.z.copy()]
    width = (hi - lo) / world
    cols[axis] = lo + width * (rank + (cols[axis] - lo) / (hi - lo))
    return Particles(cols[0], cols[1], cols[2], parts.vx, parts.vy, parts.vz, parts.species_begin, parts.q,
                     parts.m, parts.w)


class ShardedDeposit:
    """Step finalize of a sharded run: the local dG, summed over the group,
    added to every rank's G_cum."""

    def __init__(self, env: FempicEnv, group=None):
        self.env, self.group = env, group
        self.dG = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")

    def __call__(self, omega0: float, t_next: float, G_cum_out=None, G_env_out=None, stream=None):
        self.env.deposit_local(self.dG, stream=stream)
        allreduce_(self.dG, self.group)
        self.env.accumulate(omega0, t_next, self.dG, G_cum_out=G_cum_out, G_env_out=G_env_out, stream=stream)
        return self.dG
