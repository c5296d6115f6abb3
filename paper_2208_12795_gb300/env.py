"""Thin PyTorch-facing wrapper over the C ABI: device memory and streams only.

Every step of the particle path runs in the CUDA library (capi.py loads it
and raises when it is missing); this module only allocates torch tensors and
passes their device pointers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import capi
from .capi import FEMPIC_FP64, FEMPIC_MIXED, FEMPIC_MIXED_Q24  # noqa: F401


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _mesh_desc(nodes: np.ndarray, tets: np.ndarray, lo, hi) -> capi.fempic_mesh_desc:
    """Describe host arrays the caller keeps alive for the duration of the call."""
    desc = capi.fempic_mesh_desc()
    desc.n_nodes, desc.n_tets = nodes.shape[0], tets.shape[0]
    desc.nodes_xyz, desc.tet_nodes = nodes.ctypes.data, tets.ctypes.data
    for a in range(3):
        desc.bbox_lo[a], desc.bbox_hi[a] = float(lo[a]), float(hi[a])
    return desc


class ParticleState:
    """Particle SoA on the device: x, y, z (f64), vx, vy, vz (f64 or f32), tet
    (i32), status (u8), n_cross (i32), plus the host species table."""

    def __init__(self, x, y, z, vx, vy, vz, species_begin, q, m, w, tet=None, track_crossings=True):
        self.x, self.y, self.z = x, y, z
        self.vx, self.vy, self.vz = vx, vy, vz
        n = x.shape[0]
        dev = x.device
        self.tet = tet if tet is not None else torch.full((n,), -1, dtype=torch.int32, device=dev)
        self.status = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.n_cross = torch.zeros(n, dtype=torch.int32, device=dev) if track_crossings else None
        self.species_begin = np.ascontiguousarray(species_begin, dtype=np.int64)
        self.q = np.ascontiguousarray(q, dtype=np.float64)
        self.m = np.ascontiguousarray(m, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)

    @classmethod
    def from_host(cls, parts, precision: int, device="cuda", track_crossings=True, pin=False):
        vdt = torch.float64 if precision == FEMPIC_FP64 else torch.float32

        def d(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
            if pin:
                t = t.pin_memory()
            return t.to(device, non_blocking=pin)

        return cls(d(parts.x, torch.float64), d(parts.y, torch.float64), d(parts.z, torch.float64),
                   d(parts.vx, vdt), d(parts.vy, vdt), d(parts.vz, vdt), parts.species_begin, parts.q,
                   parts.m, parts.w, track_crossings=track_crossings)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def cstruct(self) -> capi.fempic_particles:
        p = capi.fempic_particles()
        p.n = self.n
        p.x, p.y, p.z = _ptr(self.x), _ptr(self.y), _ptr(self.z)
        p.vx, p.vy, p.vz = _ptr(self.vx), _ptr(self.vy), _ptr(self.vz)
        p.tet, p.status, p.n_cross = _ptr(self.tet), _ptr(self.status), _ptr(self.n_cross)
        p.n_species = len(self.q)
        p.species_begin = self.species_begin.ctypes.data
        p.q, p.m, p.w = self.q.ctypes.data, self.m.ctypes.data, self.w.ctypes.data
        return p

    def empty_like(self) -> "ParticleState":
        """Second buffer of the same shape and dtypes (the sort's output)."""
        e = lambda t: None if t is None else torch.empty_like(t)
        o = ParticleState(e(self.x), e(self.y), e(self.z), e(self.vx), e(self.vy), e(self.vz),
                          self.species_begin, self.q, self.m, self.w, tet=e(self.tet),
                          track_crossings=self.n_cross is not None)
        return o

    def swap(self, other: "ParticleState"):
        """Exchange the device buffers of two states (after a sort into `other`)."""
        for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status", "n_cross"):
            a, b = getattr(self, k), getattr(other, k)
            setattr(self, k, b)
            setattr(other, k, a)

    def to_numpy(self) -> dict:
        out = {k: getattr(self, k).cpu().numpy() for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status")}
        out["n_cross"] = None if self.n_cross is None else self.n_cross.cpu().numpy()
        return out


class FempicEnv:
    """Owner of one fempic_env handle (mesh tables and edge accumulators)."""

    def __init__(self, nodes: np.ndarray, tets: np.ndarray, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                 precision: int = FEMPIC_FP64, max_crossings: int = 4096, wall_mode: int = 0):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        self._mesh = (nodes, tets, tuple(lo), tuple(hi))
        desc = _mesh_desc(*self._mesh)
        opt = capi.fempic_options(precision, max_crossings, wall_mode, 0)
        torch.cuda.init()
        self.precision = precision
        self.h = capi.fempic_env_create(desc, opt)
        counts = np.zeros(4, np.int64)
        capi.fempic_env_query(self.h, counts.ctypes.data)
        self.n_nodes, self.n_edges, self.n_faces, self.n_tets = (int(c) for c in counts)

    @classmethod
    def from_mesh(cls, mesh, **kw):
        return cls(mesh.nodes, mesh.tets, mesh.lo, mesh.hi, **kw)

    def close(self):
        if getattr(self, "h", None):
            capi.fempic_env_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dof_dtype(self):
        return torch.complex128 if self.precision == FEMPIC_FP64 else torch.complex64

    def query(self) -> dict:
        nt, ne, nf = self.n_tets, self.n_edges, self.n_faces
        out = dict(tet_nodes=np.zeros((nt, 4), np.int32), edge_nodes=np.zeros((ne, 2), np.int32),
                   face_nodes=np.zeros((nf, 3), np.int32), tet_edges=np.zeros((nt, 6), np.int32),
                   tet_faces=np.zeros((nt, 4), np.int32), tet_nbr=np.zeros((nt, 4), np.int32))
        counts = np.zeros(4, np.int64)
        capi.fempic_env_query(self.h, counts.ctypes.data, *(out[k].ctypes.data for k in
                                                            ("tet_nodes", "edge_nodes", "face_nodes",
                                                             "tet_edges", "tet_faces", "tet_nbr")))
        return out

    def locate(self, st: ParticleState, stream=None):
        capi.fempic_locate(self.h, st.cstruct(), _stream(stream))

    def push_step(self, st: ParticleState, e_dof: torch.Tensor, b_dof: torch.Tensor, amp: float, omega0: float,
                  t: float, dt: float, stream=None):
        if e_dof.dtype != self.dof_dtype or b_dof.dtype != self.dof_dtype:
            raise capi.FempicError(f"DoFs must be {self.dof_dtype} for this precision form")
        if e_dof.numel() != self.n_edges or b_dof.numel() != self.n_faces or not e_dof.is_cuda:
            raise capi.FempicError("DoF arrays must be device tensors of length n_edges / n_faces")
        vdt = torch.float64 if self.precision == FEMPIC_FP64 else torch.float32
        if st.vx.dtype != vdt:
            raise capi.FempicError(f"velocities must be {vdt} for this precision form")
        envl = capi.fempic_envelope(_ptr(e_dof), _ptr(b_dof), float(amp))
        capi.fempic_push_step(self.h, st.cstruct(), envl, omega0, t, dt, _stream(stream))

    def push_step3(self, st: ParticleState, e_levels, b_levels, weights, amp: float, omega0: float, t: float,
                   dt: float, stream=None):
        """One step with the envelope interpolated from three DoF levels
        (levels n-1, n, n+1 with their Lagrange weights at t)."""
        if len(e_levels) != 3 or len(b_levels) != 3 or len(weights) != 3:
            raise capi.FempicError("three levels and three weights are required")
        for e_dof, b_dof in zip(e_levels, b_levels):
            if e_dof.dtype != self.dof_dtype or b_dof.dtype != self.dof_dtype:
                raise capi.FempicError(f"DoFs must be {self.dof_dtype} for this precision form")
            if e_dof.numel() != self.n_edges or b_dof.numel() != self.n_faces or not e_dof.is_cuda:
                raise capi.FempicError("DoF arrays must be device tensors of length n_edges / n_faces")
        vdt = torch.float64 if self.precision == FEMPIC_FP64 else torch.float32
        if st.vx.dtype != vdt:
            raise capi.FempicError(f"velocities must be {vdt} for this precision form")
        envl = capi.fempic_envelope3()
        for k in range(3):
            envl.e_tilde[k] = _ptr(e_levels[k])
            envl.b_tilde[k] = _ptr(b_levels[k])
            envl.weight[k] = float(weights[k])
        envl.amp = float(amp)
        capi.fempic_push_step3(self.h, st.cstruct(), envl, omega0, t, dt, _stream(stream))

    def deposit(self, omega0: float, t_next: float, dG_out=None, G_cum_out=None, G_env_out=None, stream=None):
        capi.fempic_deposit(self.h, omega0, t_next, _ptr(dG_out), _ptr(G_cum_out), _ptr(G_env_out),
                            _stream(stream))

    def deposit_local(self, dG_out, stream=None):
        """This process's step deposit into dG_out (G_cum unchanged)."""
        capi.fempic_deposit_local(self.h, _ptr(dG_out), _stream(stream))

    def accumulate(self, omega0: float, t_next: float, dG, G_cum_out=None, G_env_out=None, stream=None):
        """G_cum += dG (a step deposit summed over every shard), then the outputs."""
        capi.fempic_accumulate(self.h, omega0, t_next, _ptr(dG), _ptr(G_cum_out), _ptr(G_env_out), _stream(stream))

    @property
    def deposit_on(self) -> bool:
        return getattr(self, "_deposit_on", True)

    def set_deposit(self, enable: bool):
        """Deposit on (default) or off for later push steps (tracking unchanged)."""
        capi.fempic_set_deposit(self.h, enable)
        self._deposit_on = bool(enable)

    def reset_deposit(self, stream=None):
        capi.fempic_reset_deposit(self.h, _stream(stream))

    def nodal_charge(self, st: ParticleState, stream=None) -> torch.Tensor:
        rho = torch.empty(self.n_nodes, dtype=torch.float64, device=st.x.device)
        capi.fempic_nodal_charge(self.h, st.cstruct(), _ptr(rho), _stream(stream))
        return rho

    def sort(self, st: ParticleState, scratch: ParticleState, stream=None):
        """Sort `st` by (species, tet) through `scratch`, then swap buffers so
        `st` holds the sorted particles."""
        capi.fempic_sort(self.h, st.cstruct(), scratch.cstruct(), _stream(stream))
        st.swap(scratch)

    def sort_perm(self, st: ParticleState, out: ParticleState, perm: torch.Tensor, stream=None):
        """Sorted copy of `st` in `out`; perm[q] = index in `st` of out's particle q."""
        if perm.dtype != torch.int32 or perm.numel() != st.n or not perm.is_cuda:
            raise capi.FempicError("perm must be a device int32 tensor of length n")
        capi.fempic_sort_perm(self.h, st.cstruct(), out.cstruct(), _ptr(perm), _stream(stream))

    def stats(self, stream=None) -> dict:
        out = np.zeros(4, np.int64)
        capi.fempic_stats(self.h, out.ctypes.data, _stream(stream))
        return dict(crossings=int(out[0]), frozen=int(out[1]), steps=int(out[2]), wait_timeouts=int(out[3]))

    def error_count(self, stream=None) -> tuple:
        """Synchronize and report the steps since the last call: (ok, frozen)
        where ok is False when a step left particles unadvanced."""
        rc, n = capi.fempic_error_count(self.h, _stream(stream))
        return rc == capi.FEMPIC_OK, n

    def profile(self, enable: bool):
        """Start (clearing earlier records) or stop per-kernel event timing."""
        capi.fempic_profile_enable(self.h, enable)

    def profile_read(self) -> dict:
        """Per kernel id since profile(True): summed event time (ms), number of
        library calls timed (`launches`) and kernels launched (`kernels`).
        The crossing pass ("cross") is timed inside the push bracket too."""
        ms = np.zeros(capi.FEMPIC_K_COUNT, np.float64)
        calls = np.zeros(capi.FEMPIC_K_COUNT, np.int64)
        kern = np.zeros(capi.FEMPIC_K_COUNT, np.int64)
        capi.fempic_profile_read(self.h, ms.ctypes.data, calls.ctypes.data, kern.ctypes.data)
        names = ("locate", "field", "push", "finalize", "charge", "sort", "cross", "adjoint")
        return {nm: dict(ms=float(ms[i]), launches=int(calls[i]), kernels=int(kern[i])) for i, nm in enumerate(names)}


class Downshift:
    """The downshifted integrator of Sec. III-D on an env of any form (the
    mixed forms keep velocities, envelope samples and history in FP32).

    Velocity rule with the carrier integrated analytically over each step (M
    and L weights on the newest three envelope samples) and fourth-order
    Adams-Bashforth positions; the segment is tracked and deposited by the
    env's own step.  Holds the per-tet gather tables and the particles'
    history planes ([FEMPIC_DS_PLANES, n] on the device: f64 on an FP64 env,
    f32 on a mixed one).  Velocities are at integer levels (v^n), not half
    steps.  The history follows the particle order: re-sort the set with
    `sort`, which carries the history through the same permutation
    (fempic_sort_perm, fempic_downshift_permute)."""

    def __init__(self, env: FempicEnv, n: int, device="cuda"):
        self.env = env
        self.f32 = env.precision != FEMPIC_FP64   # mixed forms: f32 velocities, samples and history
        self.h = capi.fempic_downshift_create(_mesh_desc(*env._mesh))
        dt = torch.float32 if self.f32 else torch.float64
        self.planes = torch.zeros((capi.FEMPIC_DS_PLANES, n), dtype=dt, device=device)
        self.started = False

    def close(self):
        if getattr(self, "h", None):
            capi.fempic_downshift_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sort(self, st: ParticleState, scratch: ParticleState, stream=None):
        """Sort `st` by (species, tet) through `scratch` (buffers swapped, as
        FempicEnv.sort does) and carry the history planes along; returns the
        permutation (perm[q] = index before the sort of particle q)."""
        perm = torch.empty(st.n, dtype=torch.int32, device=st.x.device)
        self.env.sort_perm(st, scratch, perm, stream=stream)
        st.swap(scratch)
        spare = getattr(self, "_spare", None)
        if spare is None or spare.shape != self.planes.shape:
            spare = torch.empty_like(self.planes)
        hin = capi.fempic_downshift_history(st.n, _ptr(self.planes), int(self.f32))
        hout = capi.fempic_downshift_history(st.n, _ptr(spare), int(self.f32))
        capi.fempic_downshift_permute(hin, hout, _ptr(perm), _stream(stream))
        self.planes, self._spare = spare, self.planes
        return perm

    def step(self, st: ParticleState, e_dof: torch.Tensor, b_dof: torch.Tensor, amp: float, omega0: float,
             t: float, dt: float, stream=None):
        """One step from t to t + dt; amp = a(t).  The first call fills the history."""
        env = self.env
        cdt, vdt = (torch.complex64, torch.float32) if self.f32 else (torch.complex128, torch.float64)
        if e_dof.dtype != cdt or b_dof.dtype != cdt:
            raise capi.FempicError(f"DoFs must be {cdt} on this env's form")
        if e_dof.numel() != env.n_edges or b_dof.numel() != env.n_faces or not e_dof.is_cuda or not b_dof.is_cuda:
            raise capi.FempicError("DoF arrays must be device tensors of length n_edges / n_faces")
        if st.vx.dtype != vdt or st.n != self.planes.shape[1]:
            raise capi.FempicError(f"velocities must be {vdt} and the history sized for this particle set")
        hist = capi.fempic_downshift_history(st.n, _ptr(self.planes), int(self.f32))
        envl = capi.fempic_envelope(_ptr(e_dof), _ptr(b_dof), float(amp))
        capi.fempic_push_step_downshift(env.h, self.h, st.cstruct(), hist, envl, omega0, t, dt,
                                        not self.started, _stream(stream))
        self.started = True
