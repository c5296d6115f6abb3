"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds no arithmetic of the particle step itself (no barycentric
coordinates, no Whitney gather, no push, no tracking, no deposit).  It only
builds what both sides consume:

* Kuhn meshes of a cube (each hex split into 6 tets along its main diagonal),
  optionally with jittered interior nodes;
* the mesh-topology numbering convention both sides derive independently
  (edges and faces numbered lexicographically by their sorted node tuples);
* prescribed field envelopes as edge/face degrees of freedom: the TE101 cavity
  mode of the unit cube (de Rham interpolation: exact edge circulations, and
  face fluxes b = (j/omega0) * (circulation of E around the face), i.e.
  Faraday's law with the e^{j omega0 t} convention of the envelope ansatz,
  Sec. III), or windowed random complex DoFs;
* particle loads (uniform Maxwellian electrons, beams, cosine-profile plasma)
  and the Gaussian envelope ramp a(t) built on the paper's modulated-Gaussian
  excitation (Sec. IV, eq. modgauss).

Physical constants are CODATA 2018.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

E_CHARGE = 1.602176634e-19      # C
M_ELECTRON = 9.1093837015e-31   # kg
C_LIGHT = 299792458.0           # m/s
SEED_BASE = 20812795

# Permutations of the axes in lexicographic order; tet id = 6*hex + perm index.
_KUHN_PERMS = list(itertools.permutations(range(3)))


# ---------------------------------------------------------------------------
# Mesh
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Mesh:
    nodes: np.ndarray        # [Nn, 3] float64
    tets: np.ndarray         # [Nt, 4] int32, node order of the Kuhn path
    lo: np.ndarray           # [3] float64 bounding box
    hi: np.ndarray           # [3] float64
    n_cells: int             # hexes per axis
    h: float                 # hex spacing

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def kuhn_cube_mesh(n: int, jitter: float = 0.0, rng: np.random.Generator | None = None,
                   length: float = 1.0) -> Mesh:
    """Cube [0, length]^3 as n^3 hexes, each split into 6 Kuhn tets.

    Node index = i + (n+1)*(j + (n+1)*k) (x fastest).  For permutation
    pi of (x, y, z) the tet is the monotone lattice path v0 = corner,
    v1 = v0 + h e_pi0, v2 = v1 + h e_pi1, v3 = v2 + h e_pi2; the 6 paths tile
    the hex and the split is conforming between hexes.  `jitter` moves
    interior nodes by U(-jitter*h, +jitter*h) per coordinate; boundary nodes
    stay put so the walls remain planar.
    """
    h = length / n
    m = n + 1
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    # x fastest: flatten in (k, j, i) order
    idx = (ii + m * (jj + m * kk))
    nodes = np.zeros((m ** 3, 3), dtype=np.float64)
    nodes[idx.ravel(), 0] = ii.ravel() * h
    nodes[idx.ravel(), 1] = jj.ravel() * h
    nodes[idx.ravel(), 2] = kk.ravel() * h
    if jitter > 0.0:
        assert rng is not None
        interior = np.all((nodes > 0.5 * h) & (nodes < length - 0.5 * h), axis=1)
        disp = rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), 3))
        nodes[interior] += disp

    hi_, hj, hk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi_ = hi_.transpose(2, 1, 0).ravel()   # hex linear index x fastest
    hj = hj.transpose(2, 1, 0).ravel()
    hk = hk.transpose(2, 1, 0).ravel()
    n_hex = n ** 3
    tets = np.zeros((n_hex, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_KUHN_PERMS):
        c = np.stack([hi_, hj, hk], axis=1)
        verts = [c.copy()]
        for ax in perm:
            c = c.copy()
            c[:, ax] += 1
            verts.append(c)
        for v, cc in enumerate(verts):
            tets[:, p, v] = cc[:, 0] + m * (cc[:, 1] + m * cc[:, 2])
    tets = tets.reshape(n_hex * 6, 4).astype(np.int32)
    return Mesh(nodes=nodes, tets=tets, lo=np.zeros(3), hi=np.full(3, length),
                n_cells=n, h=h)


def kuhn_counts(n: int) -> dict:
    """Closed-form entity counts of the n^3 x 6 Kuhn cube."""
    nn = (n + 1) ** 3
    ne = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    nt = 6 * n ** 3
    nf = 1 - nn + ne + nt          # Euler: Nn - Ne + Nf - Nt = 1
    return dict(n_nodes=nn, n_edges=ne, n_faces=nf, n_tets=nt, n_boundary_faces=12 * n * n)


# ---------------------------------------------------------------------------
# Topology numbering convention (shared by definition, derived on both sides)
# ---------------------------------------------------------------------------
_LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
_LOCAL_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))   # face k is opposite node k


def mesh_topology(tets: np.ndarray):
    """Edges [Ne,2] and faces [Nf,3] numbered lexicographically by sorted node
    tuples, plus per-tet local->global maps for sorted tet node order.

    Returns (tet_sorted [Nt,4], edges [Ne,2], faces [Nf,3], tet_edges [Nt,6],
    tet_faces [Nt,4]).  Local edge e of a tet joins sorted local nodes
    _LOCAL_EDGES[e]; local face k is opposite sorted local node k.
    """
    ts = np.sort(tets.astype(np.int64), axis=1)
    ekeys = np.stack([ts[:, list(p)] for p in _LOCAL_EDGES], axis=1).reshape(-1, 2)
    edges, einv = np.unique(ekeys, axis=0, return_inverse=True)
    fkeys = np.stack([ts[:, list(f)] for f in _LOCAL_FACES], axis=1).reshape(-1, 3)
    faces, finv = np.unique(fkeys, axis=0, return_inverse=True)
    nt = ts.shape[0]
    return (ts.astype(np.int32), edges.astype(np.int32), faces.astype(np.int32),
            einv.reshape(nt, 6).astype(np.int32), finv.reshape(nt, 4).astype(np.int32))


# ---------------------------------------------------------------------------
# Prescribed envelopes (edge / face DoFs)
# ---------------------------------------------------------------------------
def te101_omega0(a: float = 1.0, d: float = 1.0) -> float:
    """Resonant angular frequency of the TE101 mode of an a x b x d box."""
    return C_LIGHT * math.pi * math.sqrt(1.0 / a ** 2 + 1.0 / d ** 2)


def _int_cos(alpha, beta):
    """Closed form of int_0^1 cos(alpha + beta s) ds (stable for beta -> 0)."""
    return np.cos(alpha + 0.5 * beta) * np.sinc(beta / (2.0 * math.pi))


def te101_edge_circulation(p0: np.ndarray, p1: np.ndarray, e0: float) -> np.ndarray:
    """Exact line integral of E = y_hat * e0 sin(pi x) sin(pi z) along p0->p1.

    sin A sin B = (cos(A-B) - cos(A+B))/2 and int_0^1 cos(alpha+beta s) ds
    are closed forms, so the edge DoF is exact to rounding.
    """
    d = p1 - p0
    pi = math.pi
    a1 = pi * (p0[:, 0] - p0[:, 2]); b1 = pi * (d[:, 0] - d[:, 2])
    a2 = pi * (p0[:, 0] + p0[:, 2]); b2 = pi * (d[:, 0] + d[:, 2])
    return e0 * d[:, 1] * 0.5 * (_int_cos(a1, b1) - _int_cos(a2, b2))


def face_circulation(faces: np.ndarray, edges: np.ndarray, edge_vals: np.ndarray) -> np.ndarray:
    """Circulation of edge values around each face (i<j<k): e_ij + e_jk - e_ik.

    This is the boundary of the oriented face [i, j, k] whose normal is
    (x_j - x_i) x (x_k - x_i).
    """
    n_nodes = int(max(edges.max(), faces.max())) + 1
    key = edges[:, 0].astype(np.int64) * n_nodes + edges[:, 1]
    order = np.argsort(key)
    skey = key[order]

    def eid(a, b):
        k = a.astype(np.int64) * n_nodes + b
        pos = np.searchsorted(skey, k)
        assert np.all(skey[pos] == k)
        return order[pos]

    i, j, k = faces[:, 0], faces[:, 1], faces[:, 2]
    return edge_vals[eid(i, j)] + edge_vals[eid(j, k)] - edge_vals[eid(i, k)]


def te101_dofs(nodes: np.ndarray, edges: np.ndarray, faces: np.ndarray, e0: float,
               omega0: float):
    """Complex envelope DoFs of the TE101 mode: (e_tilde [Ne], b_tilde [Nf]).

    e_tilde = exact edge circulations of E (real); b_tilde = (j/omega0) times
    the face circulation of e_tilde, which by Stokes is the exact face flux of
    B = (j/omega0) curl E.
    """
    circ = te101_edge_circulation(nodes[edges[:, 0]], nodes[edges[:, 1]], e0)
    e_t = circ.astype(np.complex128)
    b_t = (1j / omega0) * face_circulation(faces, edges, circ)
    return e_t, b_t.astype(np.complex128)


def random_windowed_dofs(nodes, edges, faces, rng, center=(0.5, 0.5, 0.5), width=0.25,
                         e_scale=1.0, b_scale=1.0):
    """Unit-variance complex normal DoFs times exp(-|x_mid - c|^2 / (2 w^2)),
    times e_scale (edges) or b_scale (faces)."""
    c = np.asarray(center, dtype=np.float64)

    def draw(n):
        return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2.0)

    em = 0.5 * (nodes[edges[:, 0]] + nodes[edges[:, 1]])
    fm = (nodes[faces[:, 0]] + nodes[faces[:, 1]] + nodes[faces[:, 2]]) / 3.0
    we = np.exp(-np.sum((em - c) ** 2, axis=1) / (2 * width ** 2))
    wf = np.exp(-np.sum((fm - c) ** 2, axis=1) / (2 * width ** 2))
    e_t = e_scale * draw(edges.shape[0]) * we
    b_t = b_scale * draw(faces.shape[0]) * wf
    return e_t.astype(np.complex128), b_t.astype(np.complex128)


def envelope_ramp(t: float, sigma: float, centered: bool = False) -> float:
    """Slow amplitude a(t) of the prescribed envelope.

    The paper's excitation (Sec. IV, eq. modgauss) is a carrier times
    exp(-(t - 6 sigma)^2 / (2 sigma^2)).  Default reading: a half-Gaussian
    rise peaking at 3 sigma and held at 1 afterwards; `centered=True` gives
    the literal 6-sigma-centred pulse.
    """
    if centered:
        return math.exp(-((t - 6.0 * sigma) ** 2) / (2.0 * sigma ** 2))
    if t < 3.0 * sigma:
        return math.exp(-((t - 3.0 * sigma) ** 2) / (2.0 * sigma ** 2))
    return 1.0


# ---------------------------------------------------------------------------
# Particle loads
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Particles:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    species_begin: np.ndarray   # int64 [n_species + 1]
    q: np.ndarray               # float64 [n_species]
    m: np.ndarray
    w: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subset(self, k: int) -> "Particles":
        """First k particles (species ranges clipped)."""
        sb = np.minimum(self.species_begin, k)
        return Particles(self.x[:k].copy(), self.y[:k].copy(), self.z[:k].copy(),
                         self.vx[:k].copy(), self.vy[:k].copy(), self.vz[:k].copy(),
                         sb.astype(np.int64), self.q.copy(), self.m.copy(), self.w.copy())


def thermal_sigma(temp_ev: float, mass: float) -> float:
    """Per-component Maxwellian velocity spread sqrt(k T / m) for T in eV."""
    return math.sqrt(E_CHARGE * temp_ev / mass)


def uniform_maxwellian(n: int, temp_ev: float, rng, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                       q=-E_CHARGE, m=M_ELECTRON, w=1e3) -> Particles:
    lo = np.asarray(lo, dtype=np.float64); hi = np.asarray(hi, dtype=np.float64)
    pos = lo + (hi - lo) * rng.random((n, 3))
    vel = rng.standard_normal((n, 3)) * thermal_sigma(temp_ev, m)
    return Particles(pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy(),
                     vel[:, 0].copy(), vel[:, 1].copy(), vel[:, 2].copy(),
                     np.array([0, n], dtype=np.int64), np.array([q]), np.array([m]),
                     np.array([w]))


def concat_species(parts: list[Particles]) -> Particles:
    """Stack single- or multi-species loads into contiguous species ranges."""
    begins = [0]
    qs, ms, ws = [], [], []
    for p in parts:
        for s in range(len(p.q)):
            begins.append(begins[-1] + int(p.species_begin[s + 1] - p.species_begin[s]))
            qs.append(p.q[s]); ms.append(p.m[s]); ws.append(p.w[s])
    cat = lambda a: np.concatenate([getattr(p, a) for p in parts])
    return Particles(cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"),
                     np.array(begins, dtype=np.int64), np.array(qs), np.array(ms), np.array(ws))


def electron_beam(n: int, energy_ev: float, spread: float, radius: float, rng,
                  center=(0.5, 0.5), w=1e3) -> Particles:
    """Electron beam along +z: Gaussian transverse profile (resampled into the
    unit cube), z uniform, non-relativistic speed sqrt(2E/m) with a Gaussian
    relative energy spread."""
    xy = np.empty((n, 2))
    filled = 0
    while filled < n:
        cand = np.asarray(center) + radius * rng.standard_normal((2 * (n - filled) + 16, 2))
        ok = cand[np.all((cand > 0.0) & (cand < 1.0), axis=1)]
        take = min(n - filled, ok.shape[0])
        xy[filled:filled + take] = ok[:take]
        filled += take
    z = rng.random(n)
    en = energy_ev * (1.0 + spread * rng.standard_normal(n))
    vz = np.sqrt(2.0 * np.maximum(en, 0.0) * E_CHARGE / M_ELECTRON)
    zeros = np.zeros(n)
    return Particles(xy[:, 0].copy(), xy[:, 1].copy(), z, zeros.copy(), zeros.copy(), vz,
                     np.array([0, n], dtype=np.int64), np.array([-E_CHARGE]),
                     np.array([M_ELECTRON]), np.array([w]))


def cosine_plasma(n: int, temp_ev: float, depth: float, rng, w=1e3) -> Particles:
    """Electrons with density proportional to 1 + depth*cos(2 pi x) (rejection
    sampled), Maxwellian at temp_ev."""
    xs = np.empty(n)
    filled = 0
    while filled < n:
        cand = rng.random(2 * (n - filled) + 16)
        acc = rng.random(cand.shape[0]) * (1.0 + depth) < 1.0 + depth * np.cos(2 * math.pi * cand)
        ok = cand[acc]
        take = min(n - filled, ok.shape[0])
        xs[filled:filled + take] = ok[:take]
        filled += take
    yz = rng.random((n, 2))
    vel = rng.standard_normal((n, 3)) * thermal_sigma(temp_ev, M_ELECTRON)
    return Particles(xs, yz[:, 0].copy(), yz[:, 1].copy(), vel[:, 0].copy(), vel[:, 1].copy(),
                     vel[:, 2].copy(), np.array([0, n], dtype=np.int64), np.array([-E_CHARGE]),
                     np.array([M_ELECTRON]), np.array([w]))


# ---------------------------------------------------------------------------
# Workloads (the five cavity / plasma cases and small test cases)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    particles: Particles
    e_tilde: np.ndarray       # complex128 [Ne]
    b_tilde: np.ndarray       # complex128 [Nf]
    omega0: float
    dt: float
    steps: int
    ramp_sigma: float         # envelope ramp sigma (s); 0 -> constant amplitude 1
    wall_mode: int = 0        # 0 reflect, 1 absorb

    def amp(self, t: float) -> float:
        return 1.0 if self.ramp_sigma <= 0.0 else envelope_ramp(t, self.ramp_sigma)


def te101_cavity(n_cells: int, n_particles: int, temp_ev: float, e0: float, steps: int,
                 seed_index: int, dt: float = 0.5e-9, ramp_sigma: float = 20e-9,
                 name: str = "", jitter: float = 0.0, wall_mode: int = 0) -> Workload:
    """Unit-cube TE101 cavity with a uniform Maxwellian electron load."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    mesh = kuhn_cube_mesh(n_cells, jitter=jitter, rng=rng)
    _, edges, faces, _, _ = mesh_topology(mesh.tets)
    om = te101_omega0()
    e_t, b_t = te101_dofs(mesh.nodes, edges, faces, e0, om)
    parts = uniform_maxwellian(n_particles, temp_ev, rng)
    return Workload(name or f"te101_{n_cells}^3x6_{n_particles}e", mesh, parts, e_t, b_t, om,
                    dt, steps, ramp_sigma, wall_mode)


def workload_hot_small(jitter: float = 0.2, wall_mode: int = 0, n_particles: int = 600,
                       steps: int = 40) -> Workload:
    """Stress case for tracking: jittered 4^3 x 6 cube, 300 eV electrons and a
    20 ns step, so most steps cross several faces and many hit a wall."""
    return te101_cavity(4, n_particles, 300.0, 1e3, steps, 11, dt=20e-9, ramp_sigma=0.0,
                        name="cube4j_hot", jitter=jitter, wall_mode=wall_mode)


def workload_small() -> Workload:
    """4^3 x 6 cube (384 tets), 2000 electrons at 1 eV, TE101 at 1 kV/m, 200 steps."""
    return te101_cavity(4, 2000, 1.0, 1e3, 200, 1, name="cube4_2k_te101")


def workload_cavity48(n_particles: int = 10_000_000) -> Workload:
    """48^3 x 6 cube (663,552 tets), 10M electrons at 5 eV, TE101 at 10 kV/m, 100 steps."""
    return te101_cavity(48, n_particles, 5.0, 1e4, 100, 2, name="cube48_10M_te101")


def RANDOM_DOF_UNITS(h: float) -> dict:
    """Units of the random envelope DoFs: unit variance in 10 kV/m x h per edge
    circulation and 10 mT x h^2 per face flux, i.e. fields of order 10 kV/m
    and 10 mT (a literal unit-variance flux on h = 1/64 would be ~4000 T)."""
    return dict(e_scale=1e4 * h, b_scale=1e-2 * h * h)


def workload_jittered64(n_particles: int = 50_000_000) -> Workload:
    """64^3 x 6 jittered cube, 10% 10 keV beam + 90% cosine plasma, random DoFs, 50 steps."""
    rng = np.random.default_rng(SEED_BASE + 3)
    mesh = kuhn_cube_mesh(64, jitter=0.2, rng=rng)
    _, edges, faces, _, _ = mesh_topology(mesh.tets)
    e_t, b_t = random_windowed_dofs(mesh.nodes, edges, faces, rng, **RANDOM_DOF_UNITS(mesh.h))
    nb = n_particles // 10
    parts = concat_species([electron_beam(nb, 1e4, 0.005, 0.1, rng),
                            cosine_plasma(n_particles - nb, 5.0, 0.5, rng)])
    return Workload("cube64j_beam_plasma", mesh, parts, e_t, b_t, te101_omega0(), 0.5e-9, 50, 0.0)


def workload_adjoint48(n_particles: int = 4_000_000) -> Workload:
    """48^3 x 6 cube, 4M electrons at 5 eV, TE101 at 10 kV/m, K = 50 steps."""
    return te101_cavity(48, n_particles, 5.0, 1e4, 50, 4, name="cube48_4M_adjoint")


def maxwellian_chunk(seed: int, chunk: int, n: int, temp_ev: float, mass: float):
    """Chunk `chunk` (n particles) of a uniform Maxwellian load, reproducible
    from (seed, chunk) alone so a very large load can be generated chunk by
    chunk: returns x, y, z, vx, vy, vz (float64)."""
    rng = np.random.default_rng([seed, chunk])
    pos = rng.random((n, 3))
    vel = rng.standard_normal((n, 3)) * thermal_sigma(temp_ev, mass)
    return pos[:, 0], pos[:, 1], pos[:, 2], vel[:, 0], vel[:, 1], vel[:, 2]


def large96_species(n_particles: int = 400_000_000):
    """Species table of the 96^3 two-species load: electrons then ions
    (m = 1836 m_e, q = +e), both at 2 eV, weight 1e3, half each."""
    half = n_particles // 2
    return (np.array([0, half, n_particles], np.int64), np.array([-E_CHARGE, E_CHARGE]),
            np.array([M_ELECTRON, 1836.0 * M_ELECTRON]), np.array([1e3, 1e3]), 2.0)


def workload_large96(n_particles: int = 400_000_000) -> Workload:
    """96^3 x 6 cube, electrons + heavy ions (m = 1836 m_e) at 2 eV, random DoFs, 20 steps."""
    rng = np.random.default_rng(SEED_BASE + 5)
    mesh = kuhn_cube_mesh(96)
    _, edges, faces, _, _ = mesh_topology(mesh.tets)
    e_t, b_t = random_windowed_dofs(mesh.nodes, edges, faces, rng, **RANDOM_DOF_UNITS(mesh.h))
    half = n_particles // 2
    el = uniform_maxwellian(half, 2.0, rng)
    ion = uniform_maxwellian(n_particles - half, 2.0, rng, q=E_CHARGE, m=1836.0 * M_ELECTRON)
    return Workload("cube96_400M_two_species", mesh, concat_species([el, ion]), e_t, b_t,
                    te101_omega0(), 0.5e-9, 20, 0.0)


# ---------------------------------------------------------------------------
# Device-side draws of the two largest loads (benchmark legs): the same
# distributions as electron_beam / cosine_plasma / uniform_maxwellian, drawn
# with a seeded torch generator on the device so that 50M-400M particles
# take seconds instead of minutes of host time.  The random numbers differ
# from the host generators'; the parity tests use the host generators.
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def device_beam_plasma(n_particles: int, seed: int, device="cuda"):
    """10% 10 keV electron beam along z (Gaussian transverse profile of radius
    0.1 about (0.5, 0.5), resampled into the cube; 0.5% energy spread) + 90%
    plasma electrons at 5 eV with density 1 + 0.5 cos(2 pi x).  Returns
    (x, y, z, vx, vy, vz) float64 device tensors and the species table."""
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = dict(dtype=torch.float64, device=device)
    nb = n_particles // 10
    npl = n_particles - nb
    # beam: transverse Gaussian, out-of-cube draws redrawn
    xy = torch.empty((nb, 2), **f64)
    todo = torch.arange(nb, device=device)
    while todo.numel():
        cand = 0.5 + 0.1 * torch.randn((todo.numel(), 2), generator=g, **f64)
        ok = ((cand > 0.0) & (cand < 1.0)).all(1)
        xy[todo[ok]] = cand[ok]
        todo = todo[~ok]
    zb = torch.rand(nb, generator=g, **f64)
    en = 1e4 * (1.0 + 0.005 * torch.randn(nb, generator=g, **f64))
    vzb = torch.sqrt(2.0 * en.clamp(min=0.0) * E_CHARGE / M_ELECTRON)
    # plasma: x by rejection against 1 + 0.5 cos(2 pi x)
    xp = torch.empty(npl, **f64)
    todo = torch.arange(npl, device=device)
    while todo.numel():
        cand = torch.rand(todo.numel(), generator=g, **f64)
        acc = torch.rand(todo.numel(), generator=g, **f64) * 1.5 < 1.0 + 0.5 * torch.cos(2 * math.pi * cand)
        xp[todo[acc]] = cand[acc]
        todo = todo[~acc]
    yzp = torch.rand((npl, 2), generator=g, **f64)
    vp = torch.randn((npl, 3), generator=g, **f64) * thermal_sigma(5.0, M_ELECTRON)
    zeros = torch.zeros(nb, **f64)
    cols = (torch.cat([xy[:, 0], xp]), torch.cat([xy[:, 1], yzp[:, 0]]), torch.cat([zb, yzp[:, 1]]),
            torch.cat([zeros, vp[:, 0]]), torch.cat([zeros, vp[:, 1]]), torch.cat([vzb, vp[:, 2]]))
    table = (np.array([0, nb, n_particles], np.int64), np.array([-E_CHARGE, -E_CHARGE]),
             np.array([M_ELECTRON, M_ELECTRON]), np.array([1e3, 1e3]))
    return cols, table


def device_two_species(n_particles: int, seed: int, device="cuda", vdtype=None):
    """Uniform electrons then heavy ions (m = 1836 m_e, q = +e), both at 2 eV,
    half each (the species table of large96_species).  Velocities in vdtype
    (float64 by default) to keep the device footprint of 400M particles low."""
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    vdtype = vdtype or torch.float64
    sb, q, m, w, temp = large96_species(n_particles)
    pos = [torch.rand(n_particles, generator=g, dtype=torch.float64, device=device) for _ in range(3)]
    vel = [torch.empty(n_particles, dtype=vdtype, device=device) for _ in range(3)]
    chunk = 50_000_000
    for s in range(2):
        sig = thermal_sigma(temp, m[s])
        for c0 in range(int(sb[s]), int(sb[s + 1]), chunk):
            c1 = min(int(sb[s + 1]), c0 + chunk)
            for k in range(3):
                vel[k][c0:c1] = (torch.randn(c1 - c0, generator=g, dtype=torch.float64, device=device) * sig).to(vdtype)
    return tuple(pos) + tuple(vel), (sb, q, m, w)
