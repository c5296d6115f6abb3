"""Gradients of a loss of K particle steps (reverse mode): the kinetic
energy after the steps, or a weighted sum of the edge current they deposit.

Every derivative is computed by the library's kernels
(`fempic_push_step_adjoint`, `fempic_kinetic_energy`,
`fempic_adjoint_current_weights`); this module only
schedules them: a forward pass that keeps a checkpoint of the particle state
every `every` steps, then a reverse sweep that, segment by segment from the
last, recomputes the segment's states from its checkpoint and runs the adjoint
steps backwards.  Memory: one state per checkpoint plus `every` + 1 states for
the segment being reversed, or 2 when the schedule does not stash (each
step's states are then recomputed from the checkpoint); `plan_window` picks
the interval and the mode for a memory budget.

Each checkpoint is taken after sorting the state by (species, tet)
(`fempic_sort_perm`), so the steps of every segment run on tet-ordered
particles; the reverse sweep carries the adjoint back across each of those
sorts with `fempic_adjoint_unpermute`.  The gradient is returned in the
particle order of the initial state.  For the kinetic energy the window's
steps run with the deposit off (`fempic_set_deposit`): that loss does not
depend on the deposited charge.  For the current loss the forward steps
deposit and each step's deposit is taken out with `fempic_deposit_local`.
Either way the env's accumulated deposit is left untouched.

The derivative is that of the piecewise smooth map for the tet sequence the
forward run took (a particle that crosses a face keeps the crossing; a
perturbation that would change the sequence is outside what it describes).
Complex DoF gradients follow dL/dRe + j dL/dIm, the convention torch uses for
real losses of complex tensors.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import capi
from .capi import FEMPIC_FP64
from .env import FempicEnv, ParticleState, _ptr, _stream


class AdjointState:
    """Adjoint of the particle state: rbar (f64) and vbar (velocity dtype)."""

    def __init__(self, n: int, vdtype, device="cuda"):
        z = lambda dt: torch.zeros(n, dtype=dt, device=device)
        self.rx, self.ry, self.rz = z(torch.float64), z(torch.float64), z(torch.float64)
        self.vx, self.vy, self.vz = z(vdtype), z(vdtype), z(vdtype)
        self.n = n

    def swap(self, other: "AdjointState"):
        for k in ("rx", "ry", "rz", "vx", "vy", "vz"):
            a, b = getattr(self, k), getattr(other, k)
            setattr(self, k, b)
            setattr(other, k, a)

    def cstruct(self) -> capi.fempic_adjoint:
        a = capi.fempic_adjoint()
        a.n = self.n
        a.rx, a.ry, a.rz = _ptr(self.rx), _ptr(self.ry), _ptr(self.rz)
        a.vx, a.vy, a.vz = _ptr(self.vx), _ptr(self.vy), _ptr(self.vz)
        return a


def clone_state(st: ParticleState) -> ParticleState:
    c = lambda t: None if t is None else t.clone()
    o = ParticleState(c(st.x), c(st.y), c(st.z), c(st.vx), c(st.vy), c(st.vz), st.species_begin, st.q, st.m, st.w,
                      tet=c(st.tet), track_crossings=st.n_cross is not None)
    o.status = st.status.clone()
    if st.n_cross is not None:
        o.n_cross = st.n_cross.clone()
    return o


def _copy_state(dst: ParticleState, src: ParticleState):
    for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status", "n_cross"):
        t = getattr(src, k)
        if t is not None:
            getattr(dst, k).copy_(t)


def kinetic_energy(env: FempicEnv, st: ParticleState, seed: AdjointState | None = None, stream=None):
    """Total kinetic energy (device f64 scalar); fills `seed` with its adjoint."""
    ke = torch.empty((), dtype=torch.float64, device=st.x.device)
    capi.fempic_kinetic_energy(env.h, st.cstruct(), _ptr(ke), seed.cstruct() if seed is not None else None,
                               _stream(stream))
    return ke


@dataclasses.dataclass
class Schedule:
    """Envelope and time stepping of a gradient window."""
    amp: object            # callable t -> a(t)
    omega0: float
    dt: float
    steps: int
    every: int = 10        # checkpoint interval
    t0: float = 0.0
    stash: bool = True     # keep a segment's recomputed states (else recompute each step's from the checkpoint)


def state_nbytes(st: ParticleState) -> int:
    """Device bytes of one particle state."""
    return sum(t.numel() * t.element_size() for t in (st.x, st.y, st.z, st.vx, st.vy, st.vz, st.tet, st.status,
                                                       st.n_cross) if t is not None)


@dataclasses.dataclass
class WindowPlan:
    every: int
    stash: bool
    peak_bytes: int        # checkpoints + working states + adjoint states (the caller's st0 not counted)
    recompute_steps: int   # forward steps the reverse sweep re-runs


def plan_window(n: int, steps: int, state_bytes: int, adj_bytes: int, budget_bytes: int) -> WindowPlan:
    """Checkpoint interval and reverse mode of a gradient window that fits in
    budget_bytes of device memory with the fewest recomputed steps (ties: the
    smaller peak).  Peak: ceil(K/every) checkpoints (a state and its sort
    permutation each), then in the reverse sweep either every + 1 stashed
    states of the segment (stash) or 2 (each step's pair recomputed from the
    checkpoint, every (every + 1) / 2 steps per segment), and the adjoint
    state with its spare for the checkpoint unpermutes.  Raises
    MemoryError when even the leanest plan does not fit."""
    perm = 4 * n
    best = None
    for every in range(1, max(steps, 1) + 1):
        nck = -(-steps // every)
        segs = [min(every, steps - s * every) for s in range(nck)]
        for stash in (True, False):
            work = (every + 1) if stash else 2
            peak = nck * (state_bytes + perm) + work * state_bytes + 2 * adj_bytes
            rec = steps if stash else sum(L * (L + 1) // 2 for L in segs)
            if peak > budget_bytes:
                continue
            key = (rec, peak)
            if best is None or key < (best.recompute_steps, best.peak_bytes):
                best = WindowPlan(every, stash, peak, rec)
    if best is None:
        raise MemoryError(f"no checkpoint plan of a {steps}-step window over {n} particles fits "
                          f"{budget_bytes / 1e9:.1f} GB")
    return best


class _DepositOff:
    """The loss does not depend on the deposited charge, so the window's
    steps run with the deposit off (same trajectories, no dG work); the
    env's accumulated deposit is left as it was."""

    def __init__(self, env: FempicEnv):
        self.env = env

    def __enter__(self):
        self.prev = self.env.deposit_on
        self.env.set_deposit(False)

    def __exit__(self, *exc):
        self.env.set_deposit(self.prev)
        return False


def _step(env, st, e, b, sch: Schedule, k: int):
    t = sch.t0 + k * sch.dt
    env.push_step(st, e, b, sch.amp(t), sch.omega0, t, sch.dt)


class Checkpoint:
    """A checkpointed state and the sort that produced its order from the
    state before it (perm[q] = previous index of particle q; None: unsorted)."""

    def __init__(self, st: ParticleState, perm):
        self.st, self.perm = st, perm


class _DepositOn:
    """The window's steps deposit (for a loss of the deposited current); each
    step's deposit is taken out with fempic_deposit_local, so G_cum is left
    as it was."""

    def __init__(self, env: FempicEnv):
        self.env = env

    def __enter__(self):
        self.prev = self.env.deposit_on
        self.env.set_deposit(True)

    def __exit__(self, *exc):
        self.env.set_deposit(self.prev)
        return False


def _forward(env: FempicEnv, st0: ParticleState, e, b, sch: Schedule, sort: bool, u=None):
    st = st0 if (sort and sch.steps > 0) else clone_state(st0)
    ckpts = []
    L = None
    if u is not None:
        L = torch.zeros((), dtype=torch.float64, device=st.x.device)
        dG = torch.empty(env.n_edges, dtype=torch.float64, device=st.x.device)
    with (_DepositOn(env) if u is not None else _DepositOff(env)):
        for k in range(sch.steps):
            if k % sch.every == 0:
                if sort:
                    srt = st.empty_like()
                    perm = torch.empty(st.n, dtype=torch.int32, device=st.x.device)
                    env.sort_perm(st, srt, perm)
                    ckpts.append(Checkpoint(srt, perm))
                    st = clone_state(srt)
                else:
                    ckpts.append(Checkpoint(clone_state(st), None))
            _step(env, st, e, b, sch, k)
            if u is not None:
                env.deposit_local(dG)
                L += torch.dot(u, dG)
    return st, ckpts, L


def forward_checkpointed(env: FempicEnv, st0: ParticleState, e, b, sch: Schedule, sort: bool = True):
    """Run sch.steps steps from a copy of st0; returns (final state,
    checkpoints).  With `sort`, the state is sorted by tet at every
    checkpoint (the final state is in the last checkpoint's order)."""
    st, ckpts, _ = _forward(env, st0, e, b, sch, sort)
    return st, ckpts


def reverse_sweep(env: FempicEnv, ckpts, e, b, sch: Schedule, adj: AdjointState, group=None):
    """Propagate `adj` (adjoint of the final state) back to the initial state;
    returns the complex128 gradients of the edge and face DoFs.  With a
    process group (particles sharded over its ranks, the loss the sum of the
    ranks' losses), the DoF gradients are summed over the ranks; the
    particles' gradients stay with their rank."""
    eg = torch.zeros(env.n_edges, dtype=torch.complex128, device=e.device)
    bg = torch.zeros(env.n_faces, dtype=torch.complex128, device=b.device)
    stream = _stream(None)
    spare = None
    for s in range(len(ckpts) - 1, -1, -1):
        k0 = s * sch.every
        k1 = min(sch.steps, k0 + sch.every)

        def adjoint_step(k, before, after):
            t = sch.t0 + k * sch.dt
            envl = capi.fempic_envelope(_ptr(e), _ptr(b), float(sch.amp(t)))
            capi.fempic_push_step_adjoint(env.h, before.cstruct(), after.cstruct(), envl, sch.omega0, t,
                                          sch.dt, adj.cstruct(), _ptr(eg), _ptr(bg), stream)

        if sch.stash:
            stash = [ckpts[s].st]
            cur = clone_state(ckpts[s].st)
            with _DepositOff(env):
                for k in range(k0, k1):
                    _step(env, cur, e, b, sch, k)
                    stash.append(clone_state(cur))
            for k in range(k1 - 1, k0 - 1, -1):
                adjoint_step(k, stash[k - k0], stash[k - k0 + 1])
            del stash, cur
        else:   # two working states: each step's (before, after) pair recomputed from the checkpoint
            before, after = clone_state(ckpts[s].st), clone_state(ckpts[s].st)
            for k in range(k1 - 1, k0 - 1, -1):
                _copy_state(before, ckpts[s].st)
                with _DepositOff(env):
                    for j in range(k0, k):
                        _step(env, before, e, b, sch, j)
                    _copy_state(after, before)
                    _step(env, after, e, b, sch, k)
                adjoint_step(k, before, after)
            del before, after
        if ckpts[s].perm is not None:   # back to the order before this checkpoint's sort
            if spare is None:
                spare = AdjointState(adj.n, adj.vx.dtype, device=adj.rx.device)
            capi.fempic_adjoint_unpermute(env.h, adj.cstruct(), spare.cstruct(), _ptr(ckpts[s].perm), stream)
            adj.swap(spare)
    if group is not None:
        from .shard import allreduce_
        allreduce_(torch.view_as_real(eg), group)
        allreduce_(torch.view_as_real(bg), group)
    return eg, bg


def kinetic_energy_and_grad(env: FempicEnv, st0: ParticleState, e, b, sch: Schedule, group=None):
    """(L, dL/de, dL/db, adjoint of the initial state) for L = kinetic energy
    after sch.steps steps from st0 (st0 is not modified).  With a process
    group, L and the DoF gradients are those of the whole sharded load."""
    final, ckpts = forward_checkpointed(env, st0, e, b, sch)
    vdt = torch.float64 if env.precision == FEMPIC_FP64 else torch.float32
    adj = AdjointState(st0.n, vdt, device=st0.x.device)
    L = kinetic_energy(env, final, seed=adj)
    del final   # the reverse sweep needs the checkpoints only
    if group is not None:
        from .shard import allreduce_
        allreduce_(L.view(1), group)
    eg, bg = reverse_sweep(env, ckpts, e, b, sch, adj, group=group)
    return L, eg, bg, adj


class _CurrentWeights:
    """Adjoint steps inside the block add the gradient of sum_e u_e dG_e."""

    def __init__(self, env: FempicEnv, u):
        self.env, self.u = env, u

    def __enter__(self):
        capi.fempic_adjoint_current_weights(self.env.h, _ptr(self.u), _stream(None))

    def __exit__(self, *exc):
        capi.fempic_adjoint_current_weights(self.env.h, None, _stream(None))
        return False


def current_loss_and_grad(env: FempicEnv, st0: ParticleState, e, b, sch: Schedule, u, group=None,
                          sort: bool = True):
    """(L, dL/de, dL/db, adjoint of the initial state) for the deposited-current
    loss L = sum_e u_e (G_cum after sch.steps steps - G_cum before), i.e. the
    weights u (device f64 [Ne]) applied to the edge deposit of the window's
    steps.  The env must hold no pending step deposit (finalize it first);
    the window's deposits are taken out step by step and G_cum is left
    unchanged.  With a process group, L and the DoF gradients are those of
    the whole sharded load."""
    u = u.to(torch.float64).contiguous()
    final, ckpts, L = _forward(env, st0, e, b, sch, sort, u=u)
    del final
    vdt = torch.float64 if env.precision == FEMPIC_FP64 else torch.float32
    adj = AdjointState(st0.n, vdt, device=st0.x.device)   # the final state does not enter L
    if group is not None:
        from .shard import allreduce_
        allreduce_(L.view(1), group)
    with _CurrentWeights(env, u):
        eg, bg = reverse_sweep(env, ckpts, e, b, sch, adj, group=group)
    return L, eg, bg, adj


class KineticEnergyAfterSteps(torch.autograd.Function):
    """L = total kinetic energy after `sch.steps` particle steps, as a
    differentiable function of the envelope DoFs (e, b) and the initial
    positions and velocities.  The forward keeps checkpoints; the backward
    runs the reverse sweep on the device."""

    @staticmethod
    def forward(ctx, e, b, x, y, z, vx, vy, vz, env: FempicEnv, template: ParticleState, sch: Schedule):
        st0 = ParticleState(x.detach(), y.detach(), z.detach(), vx.detach(), vy.detach(), vz.detach(),
                            template.species_begin, template.q, template.m, template.w, tet=template.tet.clone(),
                            track_crossings=False)
        st0.status = template.status.clone()
        final, ckpts = forward_checkpointed(env, st0, e.detach(), b.detach(), sch)
        ctx.env, ctx.sch, ctx.ckpts, ctx.final = env, sch, ckpts, final
        ctx.e, ctx.b = e.detach(), b.detach()
        ctx.dtypes = (e.dtype, b.dtype)
        return kinetic_energy(env, final).clone()

    @staticmethod
    def backward(ctx, gL):
        env, sch = ctx.env, ctx.sch
        vdt = torch.float64 if env.precision == FEMPIC_FP64 else torch.float32
        adj = AdjointState(ctx.final.n, vdt, device=ctx.final.x.device)
        kinetic_energy(env, ctx.final, seed=adj)
        eg, bg = reverse_sweep(env, ctx.ckpts, ctx.e, ctx.b, sch, adj)
        g = gL.to(torch.float64)
        return ((eg * g).to(ctx.dtypes[0]), (bg * g).to(ctx.dtypes[1]),
                adj.rx * g, adj.ry * g, adj.rz * g,
                adj.vx * g.to(vdt), adj.vy * g.to(vdt), adj.vz * g.to(vdt), None, None, None)


def grad_dot(eg, bg, adj: AdjointState, de, db, tr, tv) -> float:
    """<gradient, direction> for a direction over (e, b, r0, v0) given as
    numpy arrays (de, db complex; tr, tv [n, 3])."""
    s = float(np.sum(eg.real * de.real + eg.imag * de.imag))
    s += float(np.sum(bg.real * db.real + bg.imag * db.imag))
    r = np.stack([adj.rx.cpu().numpy(), adj.ry.cpu().numpy(), adj.rz.cpu().numpy()], 1)
    v = np.stack([adj.vx.cpu().numpy(), adj.vy.cpu().numpy(), adj.vz.cpu().numpy()], 1).astype(np.float64)
    return s + float(np.sum(r * tr)) + float(np.sum(v * tv))
