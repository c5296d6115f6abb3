"""ctypes wrapper of the plain-C FP64 oracle (fempic_oracle.c).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).  Parity status
of every function is stated in fempic_oracle.c's header and pinned by
tests/test_oracle_*.py against closed forms, invariants and brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fempic_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libfempic_oracle.so")
_lock = threading.Lock()
_lib = None

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, FP64, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        lib.or_mesh_create.restype = C.c_void_p
        lib.or_mesh_create.argtypes = [C.c_int64, _d, C.c_int64, _i32, _d, _d, C.POINTER(C.c_int32)]
        lib.or_mesh_destroy.argtypes = [C.c_void_p]
        lib.or_mesh_sizes.argtypes = [C.c_void_p, _i64]
        lib.or_mesh_tables.argtypes = [C.c_void_p] + [_i32] * 6
        lib.or_bary.argtypes = [C.c_void_p, C.c_int32, _d, _d]
        lib.or_grad_bary.argtypes = [C.c_void_p, C.c_int32, _d]
        lib.or_locate_brute_one.restype = C.c_int32
        lib.or_locate_brute_one.argtypes = [C.c_void_p, _d]
        lib.or_locate.argtypes = [C.c_void_p, C.c_int64, _d, _d, _d, _i32, _u8, C.c_int32]
        lib.or_whitney1.argtypes = [C.c_void_p, C.c_int32, _d, _d]
        lib.or_whitney2.argtypes = [C.c_void_p, C.c_int32, _d, _d]
        lib.or_gather.argtypes = [C.c_void_p, C.c_int32, _d, _d, _d, _d, _d]
        lib.or_push_step.restype = C.c_int
        lib.or_push_step.argtypes = ([C.c_void_p, C.c_int64] + [_d] * 6 +
                                     [_i32, _u8, C.c_void_p, C.c_int32, _i64, _d, _d, _d, _d, _d,
                                      C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                      C.c_int32, _d, C.c_void_p])
        lib.or_push_step_jvp.restype = C.c_int
        lib.or_push_step_jvp.argtypes = ([C.c_void_p, C.c_int64] + [_d] * 6 +
                                         [_i32, _u8, C.c_void_p, C.c_int32, _i64, _d, _d, _d, _d, _d,
                                          C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                          C.c_int32, _d, _d, _d, _d, _d, C.c_void_p])
        lib.or_nodal_charge.argtypes = [C.c_void_p, C.c_int64, _d, _d, _d, _i32, C.c_int32, _i64, _d,
                                        _d, _d]
        lib.or_edge_divergence.argtypes = [C.c_void_p, _d, _d]
        lib.or_face_circulation.argtypes = [C.c_void_p, _d, _d]
        lib.or_envelope_frame.argtypes = [C.c_int64, _d, C.c_double, C.c_double, _d]
        lib.or_kinetic_energy.restype = C.c_double
        lib.or_kinetic_energy.argtypes = [C.c_int64, _d, _d, _d, C.c_void_p, C.c_int32, _i64, _d, _d]
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleMesh:
    """Mesh tables derived by the oracle from raw nodes and tets."""

    def __init__(self, nodes, tets, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        lib = _load()
        nodes = _f64(nodes)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        err = C.c_int32(0)
        self._h = lib.or_mesh_create(nodes.shape[0], nodes.reshape(-1), tets.shape[0], tets.reshape(-1),
                                     _f64(lo), _f64(hi), C.byref(err))
        if not self._h:
            raise ValueError(f"oracle mesh rejected (code {err.value})")
        sz = np.zeros(4, dtype=np.int64)
        lib.or_mesh_sizes(self._h, sz)
        self.n_nodes, self.n_edges, self.n_faces, self.n_tets = (int(v) for v in sz)
        self.lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_mesh_destroy(h)
            self._h = None

    @property
    def h(self):
        return self._h

    def tables(self):
        nt, ne, nf = self.n_tets, self.n_edges, self.n_faces
        tn = np.zeros((nt, 4), np.int32); en = np.zeros((ne, 2), np.int32)
        fn = np.zeros((nf, 3), np.int32); te = np.zeros((nt, 6), np.int32)
        tf = np.zeros((nt, 4), np.int32); nb = np.zeros((nt, 4), np.int32)
        self.lib.or_mesh_tables(self._h, tn.reshape(-1), en.reshape(-1), fn.reshape(-1), te.reshape(-1),
                                tf.reshape(-1), nb.reshape(-1))
        return dict(tet_nodes=tn, edge_nodes=en, face_nodes=fn, tet_edges=te, tet_faces=tf, tet_nbr=nb)

    def bary(self, t, r):
        lam = np.zeros(4)
        self.lib.or_bary(self._h, int(t), _f64(r), lam)
        return lam

    def grad_bary(self, t):
        g = np.zeros(12)
        self.lib.or_grad_bary(self._h, int(t), g)
        return g.reshape(4, 3)

    def whitney1(self, t, r):
        W = np.zeros(18)
        self.lib.or_whitney1(self._h, int(t), _f64(r), W)
        return W.reshape(6, 3)

    def whitney2(self, t, r):
        W = np.zeros(12)
        self.lib.or_whitney2(self._h, int(t), _f64(r), W)
        return W.reshape(4, 3)

    def gather(self, t, r, e_dof, b_dof):
        """Complex envelope fields (E~, B~) at r in tet t."""
        Et = np.zeros(6); Bt = np.zeros(6)
        e = np.ascontiguousarray(e_dof, np.complex128).view(np.float64)
        b = np.ascontiguousarray(b_dof, np.complex128).view(np.float64)
        assert e.shape[0] == 2 * self.n_edges and b.shape[0] == 2 * self.n_faces
        self.lib.or_gather(self._h, int(t), _f64(r), e, b, Et, Bt)
        return Et[:3] + 1j * Et[3:], Bt[:3] + 1j * Bt[3:]

    def locate(self, x, y, z, brute=False):
        n = len(x)
        tet = np.zeros(n, np.int32); st = np.zeros(n, np.uint8)
        self.lib.or_locate(self._h, n, _f64(x), _f64(y), _f64(z), tet, st, 1 if brute else 0)
        return tet, st

    def locate_brute_one(self, r):
        return int(self.lib.or_locate_brute_one(self._h, _f64(r)))

    def nodal_charge(self, x, y, z, tet, species_begin, q, w):
        rho = np.zeros(self.n_nodes)
        self.lib.or_nodal_charge(self._h, len(x), _f64(x), _f64(y), _f64(z),
                                 np.ascontiguousarray(tet, np.int32), len(q),
                                 np.ascontiguousarray(species_begin, np.int64), _f64(q), _f64(w), rho)
        return rho

    def edge_divergence(self, G):
        out = np.zeros(self.n_nodes)
        self.lib.or_edge_divergence(self._h, _f64(G), out)
        return out

    def face_circulation(self, v):
        out = np.zeros(self.n_faces)
        self.lib.or_face_circulation(self._h, _f64(v), out)
        return out


class OracleState:
    """Particle SoA held as FP64 numpy arrays for the oracle."""

    def __init__(self, parts, tet=None):
        self.x = _f64(parts.x).copy(); self.y = _f64(parts.y).copy(); self.z = _f64(parts.z).copy()
        self.vx = _f64(parts.vx).copy(); self.vy = _f64(parts.vy).copy(); self.vz = _f64(parts.vz).copy()
        n = self.x.shape[0]
        self.tet = np.full(n, -1, np.int32) if tet is None else np.ascontiguousarray(tet, np.int32).copy()
        self.status = np.zeros(n, np.uint8)
        self.n_cross = np.zeros(n, np.int32)
        self.species_begin = np.ascontiguousarray(parts.species_begin, np.int64)
        self.q = _f64(parts.q); self.m = _f64(parts.m); self.w = _f64(parts.w)

    @property
    def n(self):
        return self.x.shape[0]

    def copy(self):
        c = object.__new__(OracleState)
        for k, v in self.__dict__.items():
            c.__dict__[k] = v.copy() if isinstance(v, np.ndarray) else v
        return c


def push_step(mesh: OracleMesh, st: OracleState, e_dof, b_dof, amp, omega0, t, dt, dG,
              max_crossings=4096, wall_mode=0, mirror=None):
    """One oracle particle step; accumulates into dG (float64 [Ne]).  mirror
    (uint8 [n] or None) receives each particle's mirrored axes (bit ax: the
    walls mirrored that velocity component an odd number of times)."""
    e = _f64(np.ascontiguousarray(e_dof, np.complex128).view(np.float64))
    b = _f64(np.ascontiguousarray(b_dof, np.complex128).view(np.float64))
    assert dG.dtype == np.float64 and dG.flags.c_contiguous and dG.shape[0] == mesh.n_edges
    mp = None
    if mirror is not None:
        assert mirror.dtype == np.uint8 and mirror.flags.c_contiguous and mirror.shape[0] == st.n
        mp = mirror.ctypes.data_as(C.c_void_p)
    mesh.lib.or_push_step(mesh.h, st.n, st.x, st.y, st.z, st.vx, st.vy, st.vz, st.tet, st.status,
                          st.n_cross.ctypes.data_as(C.c_void_p), len(st.q), st.species_begin, st.q,
                          st.m, st.w, e, b, float(amp), float(omega0), float(t), float(dt),
                          int(max_crossings), int(wall_mode), dG, mp)


def push_step_jvp(mesh: OracleMesh, st: OracleState, e_dof, b_dof, amp, omega0, t, dt, dG, tr, tv, de, db,
                  max_crossings=4096, wall_mode=0, dGt=None):
    """One oracle step of values and forward-mode tangents.

    tr, tv: float64 [n, 3] tangents of position and velocity (updated in
    place); de, db: complex tangent DoFs; dGt (float64 [Ne] or None): the
    tangent of the step's edge deposit is added to it."""
    e = _f64(np.ascontiguousarray(e_dof, np.complex128).view(np.float64))
    b = _f64(np.ascontiguousarray(b_dof, np.complex128).view(np.float64))
    tde = _f64(np.ascontiguousarray(de, np.complex128).view(np.float64))
    tdb = _f64(np.ascontiguousarray(db, np.complex128).view(np.float64))
    assert tr.dtype == np.float64 and tr.flags.c_contiguous and tr.shape == (st.n, 3)
    assert tv.dtype == np.float64 and tv.flags.c_contiguous and tv.shape == (st.n, 3)
    mesh.lib.or_push_step_jvp(mesh.h, st.n, st.x, st.y, st.z, st.vx, st.vy, st.vz, st.tet, st.status,
                              st.n_cross.ctypes.data_as(C.c_void_p), len(st.q), st.species_begin, st.q,
                              st.m, st.w, e, b, float(amp), float(omega0), float(t), float(dt),
                              int(max_crossings), int(wall_mode), dG, tr.reshape(-1), tv.reshape(-1),
                              tde, tdb, None if dGt is None else dGt.ctypes.data_as(C.c_void_p))


def kinetic_energy_jvp(st: OracleState, tv):
    """Tangent of the total kinetic energy sum 1/2 m w |v|^2 over active particles."""
    out = 0.0
    for s in range(len(st.q)):
        a, b = int(st.species_begin[s]), int(st.species_begin[s + 1])
        act = st.tet[a:b] >= 0
        v = np.stack([st.vx[a:b], st.vy[a:b], st.vz[a:b]], 1)[act]
        out += st.m[s] * st.w[s] * float(np.sum(v * tv[a:b][act]))
    return out


def envelope_frame(G, omega0, t):
    lib = _load()
    G = _f64(G)
    out = np.zeros(2 * G.shape[0])
    lib.or_envelope_frame(G.shape[0], G, float(omega0), float(t), out)
    return out.view(np.complex128)


def kinetic_energy(st: OracleState):
    lib = _load()
    return float(lib.or_kinetic_energy(st.n, st.vx, st.vy, st.vz, st.tet.ctypes.data_as(C.c_void_p),
                                       len(st.q), st.species_begin, st.m, st.w))


def run(mesh: OracleMesh, wl, st: OracleState, steps: int, max_crossings=4096, step0: int = 0):
    """Run `steps` oracle steps of workload `wl`; returns (state, G_cum)."""
    G = np.zeros(mesh.n_edges)
    for n in range(step0, step0 + steps):
        t = n * wl.dt
        push_step(mesh, st, wl.e_tilde, wl.b_tilde, wl.amp(t), wl.omega0, t, wl.dt, G,
                  max_crossings=max_crossings, wall_mode=wl.wall_mode)
    return st, G


# ------------------------------------------------ three-level envelope
# Sec. III-A represents the field coefficients over [t_{n-1}, t_{n+1}] by
# second-order Lagrange polynomials in time; Sec. III-D's simpler particle
# scheme samples that representation at each fine step.  Reading taken: the
# basis function multiplying level k is the one equal to 1 at that level's
# own time tau_k = t_{n-1+k}, and the carrier is applied at the fine-step time
# t (E = Re{a(t) e^{j omega0 t} sum_k N_k(t) e^k}).

def lagrange3_weights(tau, t):
    """N_k(t) = prod over j != k of (t - tau_j) / (tau_k - tau_j), k = 0, 1, 2."""
    w = []
    for k in range(3):
        num, den = 1.0, 1.0
        for j in range(3):
            if j != k:
                num *= t - tau[j]
                den *= tau[k] - tau[j]
        w.append(num / den)
    return w


def envelope3(levels, weights):
    """The envelope at t: sum_k N_k(t) level_k (complex128 arrays)."""
    out = np.zeros_like(np.asarray(levels[0], dtype=np.complex128))
    for lv, wk in zip(levels, weights):
        out = out + wk * np.asarray(lv, dtype=np.complex128)
    return out


def envelope3_literal(levels, weights, tau, omega0, t):
    """The fine-step field formula with the carrier of each level's own time
    inside the interpolation (Sec. III-D as printed): the field at t is
    Re{sum_k N_k(t) level_k e^{j omega0 tau_k}}.  Returned as the envelope
    that the carrier at t turns into that field, sum_k N_k(t) level_k
    e^{j omega0 (tau_k - t)}, so that push_step takes it unchanged."""
    out = np.zeros_like(np.asarray(levels[0], dtype=np.complex128))
    for lv, wk, tk in zip(levels, weights, tau):
        out = out + (wk * np.exp(1j * omega0 * (tk - t))) * np.asarray(lv, dtype=np.complex128)
    return out


def push_step3(mesh: OracleMesh, st: OracleState, e_levels, b_levels, weights, amp, omega0, t, dt, dG,
               max_crossings=4096, wall_mode=0, tau=None, literal_phase=False):
    """One oracle step with the envelope interpolated from three levels.
    Default: the reading taken (carrier at the fine-step time t).  With
    literal_phase, the printed formula's per-level carrier e^{j omega0 tau_k}
    (tau: the three level times)."""
    if literal_phase:
        e_env = envelope3_literal(e_levels, weights, tau, omega0, t)
        b_env = envelope3_literal(b_levels, weights, tau, omega0, t)
    else:
        e_env, b_env = envelope3(e_levels, weights), envelope3(b_levels, weights)
    push_step(mesh, st, e_env, b_env, amp, omega0, t, dt, dG, max_crossings=max_crossings, wall_mode=wall_mode)
