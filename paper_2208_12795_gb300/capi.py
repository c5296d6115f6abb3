"""ctypes binding of the C ABI in include/fempic_env.h (argument marshalling only).

Function names match the C entry points.  The library is loaded from the
package directory; when it is missing the import of any entry point raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# FEMPIC_LIBRARY selects another build of the same library (the debug build,
# libfempic_env_debug.so, in the tests of its bounds checks)
LIB_PATH = os.environ.get("FEMPIC_LIBRARY") or os.path.join(HERE, "libfempic_env.so")

FEMPIC_OK = 0
FEMPIC_EINVAL = -1
FEMPIC_ECUDA = -2
FEMPIC_EMESH = -3
FEMPIC_ENOMEM = -4
FEMPIC_EINCOMPLETE = -5
FEMPIC_EBOUNDS = -6
FEMPIC_TABLE_NEIGHBOUR = 0
FEMPIC_TABLE_EDGE = 1
FEMPIC_TABLE_FACE = 2
FEMPIC_FP64 = 0
FEMPIC_MIXED = 1
FEMPIC_MIXED_Q24 = 2
FEMPIC_P_OK, FEMPIC_P_CAP, FEMPIC_P_ABSORBED, FEMPIC_P_NONFINITE, FEMPIC_P_LOST = range(5)
FEMPIC_WALL_REFLECT = 0
FEMPIC_WALL_ABSORB = 1

# Every function declared in include/fempic_env.h.
EXPORTS = ("fempic_env_create", "fempic_env_query", "fempic_locate", "fempic_push_step", "fempic_push_step3",
           "fempic_lagrange3",
           "fempic_deposit", "fempic_deposit_local", "fempic_accumulate", "fempic_reset_deposit", "fempic_set_deposit", "fempic_nodal_charge", "fempic_stats",
           "fempic_error_count", "fempic_debug_stall", "fempic_debug_set_table", "fempic_adjoint_current_weights", "fempic_push_step_adjoint", "fempic_kinetic_energy", "fempic_sort", "fempic_sort_perm",
           "fempic_adjoint_unpermute", "fempic_sort_noalloc", "fempic_profile_enable", "fempic_profile_read",
           "fempic_measure_fp64_rate", "fempic_last_error", "fempic_env_destroy")
# Every function declared in include/fempic_downshift.h.
DS_EXPORTS = ("fempic_downshift_create", "fempic_downshift_weights", "fempic_push_step_downshift",
              "fempic_downshift_permute", "fempic_downshift_last_error", "fempic_downshift_destroy",
              "fempic_downshift_debug_set_table")
FEMPIC_DS_VH, FEMPIC_DS_F, FEMPIC_DS_VN, FEMPIC_DS_U, FEMPIC_DS_PLANES = 0, 9, 33, 36, 39
FEMPIC_K_LOCATE, FEMPIC_K_FIELD, FEMPIC_K_PUSH, FEMPIC_K_FINALIZE, FEMPIC_K_CHARGE, FEMPIC_K_SORT, FEMPIC_K_CROSS, \
    FEMPIC_K_ADJOINT = range(8)
FEMPIC_K_COUNT = 8
FEMPIC_SORT_NOALLOC_MAX_KEYS = 1 << 21


class fempic_mesh_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("nodes_xyz", C.c_void_p),
                ("tet_nodes", C.c_void_p), ("bbox_lo", C.c_double * 3), ("bbox_hi", C.c_double * 3)]


class fempic_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_crossings", C.c_int32), ("wall_mode", C.c_int32),
                ("reserved", C.c_int32)]


class fempic_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p), ("tet", C.c_void_p),
                ("status", C.c_void_p), ("n_cross", C.c_void_p), ("n_species", C.c_int32),
                ("species_begin", C.c_void_p), ("q", C.c_void_p), ("m", C.c_void_p), ("w", C.c_void_p)]


class fempic_adjoint(C.Structure):
    _fields_ = [("n", C.c_int64), ("rx", C.c_void_p), ("ry", C.c_void_p), ("rz", C.c_void_p),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p)]


class fempic_envelope(C.Structure):
    _fields_ = [("e_tilde", C.c_void_p), ("b_tilde", C.c_void_p), ("amp", C.c_double)]


class fempic_envelope3(C.Structure):
    _fields_ = [("e_tilde", C.c_void_p * 3), ("b_tilde", C.c_void_p * 3), ("weight", C.c_double * 3),
                ("amp", C.c_double)]


class fempic_downshift_history(C.Structure):
    _fields_ = [("n", C.c_int64), ("planes", C.c_void_p), ("f32", C.c_int32)]


class FempicError(RuntimeError):
    pass


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FempicError(f"{path} is missing: build it with paper_2208_12795_gb300.build.build()")
        lib = C.CDLL(path)
        P = C.POINTER
        lib.fempic_env_create.argtypes = [P(fempic_mesh_desc), P(fempic_options), P(C.c_void_p)]
        lib.fempic_env_query.argtypes = [C.c_void_p] + [C.c_void_p] * 7
        lib.fempic_locate.argtypes = [C.c_void_p, P(fempic_particles), C.c_void_p]
        lib.fempic_push_step3.argtypes = [C.c_void_p, P(fempic_particles), P(fempic_envelope3), C.c_double,
                                          C.c_double, C.c_double, C.c_void_p]
        lib.fempic_lagrange3.argtypes = [C.c_void_p, C.c_double, C.c_void_p]
        lib.fempic_push_step.argtypes = [C.c_void_p, P(fempic_particles), P(fempic_envelope), C.c_double,
                                         C.c_double, C.c_double, C.c_void_p]
        lib.fempic_deposit.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
        lib.fempic_reset_deposit.argtypes = [C.c_void_p, C.c_void_p]
        lib.fempic_deposit_local.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.fempic_accumulate.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
        lib.fempic_set_deposit.argtypes = [C.c_void_p, C.c_int32]
        lib.fempic_nodal_charge.argtypes = [C.c_void_p, P(fempic_particles), C.c_void_p, C.c_void_p]
        lib.fempic_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.fempic_error_count.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.fempic_debug_stall.argtypes = [C.c_void_p, C.c_int32, C.c_int64]
        lib.fempic_debug_set_table.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int32]
        lib.fempic_adjoint_current_weights.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.fempic_push_step_adjoint.argtypes = [C.c_void_p, P(fempic_particles), P(fempic_particles),
                                                 P(fempic_envelope), C.c_double, C.c_double, C.c_double,
                                                 P(fempic_adjoint), C.c_void_p, C.c_void_p, C.c_void_p]
        lib.fempic_kinetic_energy.argtypes = [C.c_void_p, P(fempic_particles), C.c_void_p, C.c_void_p,
                                              C.c_void_p]
        lib.fempic_sort.argtypes = [C.c_void_p, P(fempic_particles), P(fempic_particles), C.c_void_p]
        lib.fempic_sort_noalloc.argtypes = [C.c_void_p, P(fempic_particles), P(fempic_particles), C.c_void_p]
        lib.fempic_sort_perm.argtypes = [C.c_void_p, P(fempic_particles), P(fempic_particles), C.c_void_p,
                                         C.c_void_p]
        lib.fempic_adjoint_unpermute.argtypes = [C.c_void_p, P(fempic_adjoint), P(fempic_adjoint), C.c_void_p,
                                                 C.c_void_p]
        lib.fempic_profile_enable.argtypes = [C.c_void_p, C.c_int32]
        lib.fempic_profile_read.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.fempic_measure_fp64_rate.argtypes = [C.c_void_p, C.c_void_p]
        lib.fempic_downshift_create.argtypes = [P(fempic_mesh_desc), P(C.c_void_p)]
        lib.fempic_downshift_weights.argtypes = [C.c_double, C.c_double, C.c_double, C.c_void_p]
        lib.fempic_push_step_downshift.argtypes = [C.c_void_p, C.c_void_p, P(fempic_particles),
                                                   P(fempic_downshift_history), P(fempic_envelope), C.c_double,
                                                   C.c_double, C.c_double, C.c_int32, C.c_void_p]
        lib.fempic_downshift_permute.argtypes = [P(fempic_downshift_history), P(fempic_downshift_history),
                                                 C.c_void_p, C.c_void_p]
        lib.fempic_downshift_last_error.restype = C.c_char_p
        lib.fempic_downshift_last_error.argtypes = []
        lib.fempic_downshift_destroy.argtypes = [C.c_void_p]
        lib.fempic_downshift_destroy.restype = None
        lib.fempic_downshift_debug_set_table.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int32]
        for name in ("fempic_downshift_create", "fempic_downshift_weights", "fempic_push_step_downshift",
                     "fempic_downshift_permute", "fempic_downshift_debug_set_table"):
            getattr(lib, name).restype = C.c_int
        lib.fempic_last_error.restype = C.c_char_p
        lib.fempic_last_error.argtypes = []
        lib.fempic_env_destroy.argtypes = [C.c_void_p]
        lib.fempic_env_destroy.restype = None
        for name in EXPORTS:
            if name not in ("fempic_last_error", "fempic_env_destroy"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def check(rc: int, what: str):
    if rc != FEMPIC_OK:
        msg = load().fempic_last_error().decode(errors="replace")
        raise FempicError(f"{what} failed ({rc}): {msg}")


# Same-named thin wrappers ------------------------------------------------
def fempic_env_create(mesh: fempic_mesh_desc, opts: fempic_options) -> int:
    h = C.c_void_p()
    check(load().fempic_env_create(C.byref(mesh), C.byref(opts), C.byref(h)), "fempic_env_create")
    return h.value


def fempic_env_query(env, counts4, tet_nodes=0, edge_nodes=0, face_nodes=0, tet_edges=0, tet_faces=0,
                     tet_nbr=0):
    check(load().fempic_env_query(env, counts4, tet_nodes, edge_nodes, face_nodes, tet_edges, tet_faces,
                                  tet_nbr), "fempic_env_query")


def fempic_locate(env, parts: fempic_particles, stream=0):
    check(load().fempic_locate(env, C.byref(parts), stream), "fempic_locate")


def fempic_push_step(env, parts: fempic_particles, envl: fempic_envelope, omega0, t, dt, stream=0):
    check(load().fempic_push_step(env, C.byref(parts), C.byref(envl), float(omega0), float(t), float(dt),
                                  stream), "fempic_push_step")


def fempic_push_step3(env, parts: fempic_particles, envl: fempic_envelope3, omega0, t, dt, stream=0):
    check(load().fempic_push_step3(env, C.byref(parts), C.byref(envl), float(omega0), float(t), float(dt),
                                   stream), "fempic_push_step3")


def fempic_lagrange3(tau, t) -> tuple:
    """Second-order Lagrange weights of the three level times tau at t."""
    tau_c = (C.c_double * 3)(*[float(x) for x in tau])
    w = (C.c_double * 3)()
    check(load().fempic_lagrange3(tau_c, float(t), w), "fempic_lagrange3")
    return tuple(w)


def fempic_set_deposit(env, enable: bool):
    check(load().fempic_set_deposit(env, 1 if enable else 0), "fempic_set_deposit")


def fempic_deposit(env, omega0, t_next, dG_out=0, G_cum_out=0, G_env_out=0, stream=0):
    check(load().fempic_deposit(env, float(omega0), float(t_next), dG_out, G_cum_out, G_env_out, stream),
          "fempic_deposit")


def fempic_deposit_local(env, dG_out, stream=0):
    check(load().fempic_deposit_local(env, dG_out, stream), "fempic_deposit_local")


def fempic_accumulate(env, omega0, t_next, dG, G_cum_out=0, G_env_out=0, stream=0):
    check(load().fempic_accumulate(env, float(omega0), float(t_next), dG, G_cum_out, G_env_out, stream),
          "fempic_accumulate")


def fempic_reset_deposit(env, stream=0):
    check(load().fempic_reset_deposit(env, stream), "fempic_reset_deposit")


def fempic_nodal_charge(env, parts: fempic_particles, rho, stream=0):
    check(load().fempic_nodal_charge(env, C.byref(parts), rho, stream), "fempic_nodal_charge")


def fempic_stats(env, out4, stream=0):
    check(load().fempic_stats(env, out4, stream), "fempic_stats")


def fempic_error_count(env, stream=0) -> tuple:
    """(return code, particles frozen since the last call); the code is
    FEMPIC_OK, FEMPIC_EINCOMPLETE or FEMPIC_EBOUNDS (any other code raises)."""
    n = C.c_int64(0)
    rc = load().fempic_error_count(env, C.byref(n), stream)
    if rc not in (FEMPIC_OK, FEMPIC_EINCOMPLETE, FEMPIC_EBOUNDS):
        check(rc, "fempic_error_count")
    return rc, n.value


def fempic_debug_stall(env, cta: int, limit_ns: int):
    check(load().fempic_debug_stall(env, int(cta), int(limit_ns)), "fempic_debug_stall")


def fempic_debug_set_table(env, table: int, index: int, value: int) -> int:
    """Return code of fempic_debug_set_table (FEMPIC_EINVAL from the release
    build); other failures raise."""
    rc = load().fempic_debug_set_table(env, int(table), int(index), int(value))
    if rc not in (FEMPIC_OK, FEMPIC_EINVAL):
        check(rc, "fempic_debug_set_table")
    return rc


def fempic_adjoint_current_weights(env, u, stream=0):
    check(load().fempic_adjoint_current_weights(env, u, stream), "fempic_adjoint_current_weights")


def fempic_push_step_adjoint(env, before: fempic_particles, after: fempic_particles, envl: fempic_envelope,
                             omega0, t, dt, adj: fempic_adjoint, e_grad, b_grad, stream=0):
    check(load().fempic_push_step_adjoint(env, C.byref(before), C.byref(after), C.byref(envl), float(omega0),
                                          float(t), float(dt), C.byref(adj), e_grad, b_grad, stream),
          "fempic_push_step_adjoint")


def fempic_kinetic_energy(env, parts: fempic_particles, ke, seed=None, stream=0):
    check(load().fempic_kinetic_energy(env, C.byref(parts), ke, C.byref(seed) if seed is not None else None,
                                       stream), "fempic_kinetic_energy")


def fempic_sort(env, parts_in: fempic_particles, parts_out: fempic_particles, stream=0):
    check(load().fempic_sort(env, C.byref(parts_in), C.byref(parts_out), stream), "fempic_sort")


def fempic_sort_perm(env, parts_in: fempic_particles, parts_out: fempic_particles, perm, stream=0):
    check(load().fempic_sort_perm(env, C.byref(parts_in), C.byref(parts_out), perm, stream), "fempic_sort_perm")


def fempic_adjoint_unpermute(env, adj_in: fempic_adjoint, adj_out: fempic_adjoint, perm, stream=0):
    check(load().fempic_adjoint_unpermute(env, C.byref(adj_in), C.byref(adj_out), perm, stream),
          "fempic_adjoint_unpermute")


def fempic_sort_noalloc(env, parts_in: fempic_particles, parts_out: fempic_particles, stream=0):
    check(load().fempic_sort_noalloc(env, C.byref(parts_in), C.byref(parts_out), stream),
          "fempic_sort_noalloc")


def fempic_profile_enable(env, enable: bool):
    check(load().fempic_profile_enable(env, 1 if enable else 0), "fempic_profile_enable")


def fempic_profile_read(env, ms_out, calls_out, kernels_out):
    check(load().fempic_profile_read(env, ms_out, calls_out, kernels_out), "fempic_profile_read")


def fempic_measure_fp64_rate(stream=0) -> float:
    r = C.c_double(0.0)
    check(load().fempic_measure_fp64_rate(C.byref(r), stream), "fempic_measure_fp64_rate")
    return r.value


def fempic_last_error() -> str:
    return load().fempic_last_error().decode(errors="replace")


def fempic_env_destroy(env):
    if env:
        load().fempic_env_destroy(env)


# Downshifted integrator (include/fempic_downshift.h) ----------------------
def check_ds(rc: int, what: str):
    if rc != FEMPIC_OK:
        msg = load().fempic_downshift_last_error().decode(errors="replace")
        raise FempicError(f"{what} failed ({rc}): {msg}")


def fempic_downshift_create(mesh: fempic_mesh_desc) -> int:
    h = C.c_void_p()
    check_ds(load().fempic_downshift_create(C.byref(mesh), C.byref(h)), "fempic_downshift_create")
    return h.value


def fempic_downshift_weights(t, dt, omega0) -> tuple:
    """(M^r[3], M^i[3], L^r[3][3], L^i[3][3]) of the step [t, t + dt]."""
    w = (C.c_double * 24)()
    check_ds(load().fempic_downshift_weights(float(t), float(dt), float(omega0), w), "fempic_downshift_weights")
    w = list(w)
    return (w[0:3], w[3:6], [w[6 + 3 * j:9 + 3 * j] for j in range(3)],
            [w[15 + 3 * j:18 + 3 * j] for j in range(3)])


def fempic_push_step_downshift(env, ds, parts: fempic_particles, hist: fempic_downshift_history,
                               envl: fempic_envelope, omega0, t, dt, start: bool, stream=0):
    check_ds(load().fempic_push_step_downshift(env, ds, C.byref(parts), C.byref(hist), C.byref(envl),
                                               float(omega0), float(t), float(dt), 1 if start else 0, stream),
             "fempic_push_step_downshift")


def fempic_downshift_permute(hist_in: fempic_downshift_history, hist_out: fempic_downshift_history, perm,
                             stream=0):
    check_ds(load().fempic_downshift_permute(C.byref(hist_in), C.byref(hist_out), perm, stream),
             "fempic_downshift_permute")


def fempic_downshift_last_error() -> str:
    return load().fempic_downshift_last_error().decode(errors="replace")


def fempic_downshift_destroy(ds):
    load().fempic_downshift_destroy(ds)


def fempic_downshift_debug_set_table(ds, table: int, index: int, value: int) -> int:
    """Return code of fempic_downshift_debug_set_table (FEMPIC_EINVAL from the
    release build); other failures raise."""
    rc = load().fempic_downshift_debug_set_table(ds, int(table), int(index), int(value))
    if rc not in (FEMPIC_OK, FEMPIC_EINVAL):
        check_ds(rc, "fempic_downshift_debug_set_table")
    return rc
