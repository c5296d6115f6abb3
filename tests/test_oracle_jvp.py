"""Pin of the oracle's forward-mode tangent (JVP) against central finite
differences of the oracle itself, for the total kinetic energy after K steps
as a function of the envelope DoFs and the initial phase space.  The tet
sequence is the same for the +h and -h runs (checked), so the loss is smooth
there and central differences are accurate to O(h^2)."""
import numpy as np
import pytest

from oracle.oracle import (OracleMesh, OracleState, kinetic_energy, kinetic_energy_jvp, push_step,
                           push_step_jvp)
from paper_2208_12795_gb300 import inputs as I


def _run(om, wl, P, tet, e, b, K, jvp=None):
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    if jvp is not None:
        tr, tv, de, db = (x.copy() for x in jvp)
    for n in range(K):
        t = n * wl.dt
        if jvp is None:
            push_step(om, st, e, b, wl.amp(t), wl.omega0, t, wl.dt, G, wall_mode=wl.wall_mode)
        else:
            push_step_jvp(om, st, e, b, wl.amp(t), wl.omega0, t, wl.dt, G, tr, tv, de, db,
                          wall_mode=wl.wall_mode)
    return st, (kinetic_energy_jvp(st, tv) if jvp is not None else None)


@pytest.mark.parametrize("maker,K", [(I.workload_small, 20), (lambda: I.workload_hot_small(n_particles=60), 6)])
def test_jvp_matches_central_differences(maker, K):
    wl = maker()
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles.subset(min(wl.particles.n, 300))
    tet, _ = om.locate(P.x, P.y, P.z)
    rng = np.random.default_rng(31)
    n = P.n
    sv = np.std(np.r_[P.vx, P.vy, P.vz])
    for trial in range(3):
        de = (rng.standard_normal(om.n_edges) + 1j * rng.standard_normal(om.n_edges)) * np.abs(wl.e_tilde).max()
        db = (rng.standard_normal(om.n_faces) + 1j * rng.standard_normal(om.n_faces)) * np.abs(wl.b_tilde).max()
        tv = rng.standard_normal((n, 3)) * sv
        tr = rng.standard_normal((n, 3)) * 1e-3 * wl.mesh.h
        base, jv = _run(om, wl, P, tet, wl.e_tilde, wl.b_tilde, K, jvp=(tr, tv, de, db))
        h = 1e-6
        outs = []
        for sgn in (1, -1):
            Pp = I.Particles(P.x + sgn * h * tr[:, 0], P.y + sgn * h * tr[:, 1], P.z + sgn * h * tr[:, 2],
                             P.vx + sgn * h * tv[:, 0], P.vy + sgn * h * tv[:, 1], P.vz + sgn * h * tv[:, 2],
                             P.species_begin, P.q, P.m, P.w)
            st, _ = _run(om, wl, Pp, tet, wl.e_tilde + sgn * h * de, wl.b_tilde + sgn * h * db, K)
            assert np.array_equal(st.tet, base.tet) and np.array_equal(st.n_cross, base.n_cross)
            outs.append(kinetic_energy(st))
        fd = (outs[0] - outs[1]) / (2 * h)
        assert abs(fd - jv) <= 1e-6 * abs(jv), (fd, jv)



def _random_dof_small():
    """The 4^3 x 6 cavity load with random windowed complex DoFs: complex
    envelope (so the carrier's imaginary part enters) and a B~ that is not
    solenoidal (so dB~/dr = beta dr does not vanish inside a tet)."""
    base = I.workload_small()
    om = OracleMesh(base.mesh.nodes, base.mesh.tets)
    tb = om.tables()
    e, b = I.random_windowed_dofs(base.mesh.nodes, tb["edge_nodes"], tb["face_nodes"], np.random.default_rng(41),
                                  e_scale=300.0, b_scale=3e-5)
    return I.Workload("cube4_random_dofs", base.mesh, base.particles, e, b, base.omega0, base.dt, 20, 0.0)


@pytest.mark.parametrize("maker,K", [(I.workload_small, 20), (lambda: I.workload_hot_small(n_particles=60), 6),
                                     (_random_dof_small, 20)])
def test_jvp_state_tangent_matches_central_differences(maker, K):
    """The tangents of every particle's final position and velocity, not only
    of the kinetic energy: the magnetic terms (dB~/dr through W2, the Boris
    rotation) do no work, so they show in the state tangent, not in the
    energy's."""
    wl = maker()
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles.subset(min(wl.particles.n, 300))
    tet, _ = om.locate(P.x, P.y, P.z)
    rng = np.random.default_rng(37)
    n = P.n
    sv = np.std(np.r_[P.vx, P.vy, P.vz])
    de = (rng.standard_normal(om.n_edges) + 1j * rng.standard_normal(om.n_edges)) * np.abs(wl.e_tilde).max()
    db = (rng.standard_normal(om.n_faces) + 1j * rng.standard_normal(om.n_faces)) * np.abs(wl.b_tilde).max()
    tv0 = rng.standard_normal((n, 3)) * sv
    tr0 = rng.standard_normal((n, 3)) * 1e-3 * wl.mesh.h
    tr, tv = tr0.copy(), tv0.copy()
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    for k in range(K):
        t = k * wl.dt
        push_step_jvp(om, st, wl.e_tilde, wl.b_tilde, wl.amp(t), wl.omega0, t, wl.dt, G, tr, tv, de, db,
                      wall_mode=wl.wall_mode)
    h = 1e-6
    outs = []
    for sgn in (1, -1):
        Pp = I.Particles(P.x + sgn * h * tr0[:, 0], P.y + sgn * h * tr0[:, 1], P.z + sgn * h * tr0[:, 2],
                         P.vx + sgn * h * tv0[:, 0], P.vy + sgn * h * tv0[:, 1], P.vz + sgn * h * tv0[:, 2],
                         P.species_begin, P.q, P.m, P.w)
        s2, _ = _run(om, wl, Pp, tet, wl.e_tilde + sgn * h * de, wl.b_tilde + sgn * h * db, K)
        assert np.array_equal(s2.tet, st.tet) and np.array_equal(s2.n_cross, st.n_cross)
        outs.append((np.stack([s2.x, s2.y, s2.z], 1), np.stack([s2.vx, s2.vy, s2.vz], 1)))
    fd_r = (outs[0][0] - outs[1][0]) / (2 * h)
    fd_v = (outs[0][1] - outs[1][1]) / (2 * h)
    assert np.abs(fd_r - tr).max() <= 1e-6 * np.abs(tr).max(), np.abs(fd_r - tr).max() / np.abs(tr).max()
    assert np.abs(fd_v - tv).max() <= 1e-6 * np.abs(tv).max(), np.abs(fd_v - tv).max() / np.abs(tv).max()


def test_jvp_values_follow_the_step_on_face_ending_segments():
    """The tangent step tracks exactly like the step: on segments that end on
    an interior face up to rounding (where the entry-face rule decides
    between one crossing and a bounce), tets, crossing counts, statuses and
    positions agree bit for bit."""
    m = I.kuhn_cube_mesh(4, jitter=0.2, rng=np.random.default_rng(7))
    om = OracleMesh(m.nodes, m.tets)
    tb = om.tables()
    nb, tn = tb["tet_nbr"], tb["tet_nodes"]
    rng = np.random.default_rng(6)
    dt = 1e-9
    xs, vs = [], []
    for t in range(om.n_tets):
        for k in range(4):
            if nb[t, k] < 0:
                continue
            X = m.nodes[[tn[t, i] for i in range(4) if i != k]]
            inner = m.nodes[tn[t]].mean(0)
            for _ in range(2):
                b = rng.dirichlet(np.ones(3)) @ X
                a = b + (inner - b) * rng.uniform(0.05, 0.5)
                xs.append(a); vs.append((b - a) / dt)
    xs, vs = np.array(xs), np.array(vs)
    n = len(xs)
    P = I.Particles(*(np.ascontiguousarray(c) for c in (xs[:, 0], xs[:, 1], xs[:, 2], vs[:, 0], vs[:, 1], vs[:, 2])),
                    np.array([0, n], np.int64), np.array([-I.E_CHARGE]), np.array([I.M_ELECTRON]), np.array([1.0]))
    tet, _ = om.locate(P.x, P.y, P.z)
    ze, zb = np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex)
    s1 = OracleState(P, tet)
    push_step(om, s1, ze, zb, 1.0, 0.0, 0.0, dt, np.zeros(om.n_edges), max_crossings=16)
    s2 = OracleState(P, tet)
    tr, tv = np.zeros((n, 3)), np.ones((n, 3))
    push_step_jvp(om, s2, ze, zb, 1.0, 0.0, 0.0, dt, np.zeros(om.n_edges), tr, tv, ze, zb, max_crossings=16)
    assert (s1.n_cross == 1).sum() > n // 10
    for k in ("tet", "n_cross", "status", "x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(getattr(s1, k), getattr(s2, k)), k


@pytest.mark.parametrize("maker,K,wall", [(lambda: I.workload_hot_small(n_particles=60), 5, 0),
                                          (lambda: I.workload_hot_small(n_particles=60, wall_mode=1), 5, 1),
                                          (I.workload_small, 15, 0)])
def test_deposit_tangent_matches_central_differences(maker, K, wall):
    """The tangent of the accumulated edge deposit G after K steps (pieces
    split at crossings, wall reflections, absorption): every edge's value
    against central differences of the oracle's own deposit, with the tet
    sequence held (checked) so that G is smooth between the two runs."""
    wl = maker()
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles
    tet, _ = om.locate(P.x, P.y, P.z)
    rng = np.random.default_rng(61)
    n = P.n
    sv = np.std(np.r_[P.vx, P.vy, P.vz])

    def run(Pp, e, b, jvp=None):
        st = OracleState(Pp, tet)
        G = np.zeros(om.n_edges)
        dGt = np.zeros(om.n_edges)
        if jvp is not None:
            tr, tv, de, db = (x.copy() for x in jvp)
        for k in range(K):
            t = k * wl.dt
            if jvp is None:
                push_step(om, st, e, b, wl.amp(t), wl.omega0, t, wl.dt, G, wall_mode=wall)
            else:
                push_step_jvp(om, st, e, b, wl.amp(t), wl.omega0, t, wl.dt, G, tr, tv, de, db, wall_mode=wall,
                              dGt=dGt)
        return st, G, dGt

    for trial in range(3):
        de = (rng.standard_normal(om.n_edges) + 1j * rng.standard_normal(om.n_edges)) * np.abs(wl.e_tilde).max()
        db = (rng.standard_normal(om.n_faces) + 1j * rng.standard_normal(om.n_faces)) * np.abs(wl.b_tilde).max()
        tv = rng.standard_normal((n, 3)) * sv
        tr = rng.standard_normal((n, 3)) * 1e-3 * wl.mesh.h
        base, G0, dGt = run(P, wl.e_tilde, wl.b_tilde, jvp=(tr, tv, de, db))
        h = 1e-7
        Gs = []
        for sgn in (1, -1):
            Pp = I.Particles(P.x + sgn * h * tr[:, 0], P.y + sgn * h * tr[:, 1], P.z + sgn * h * tr[:, 2],
                             P.vx + sgn * h * tv[:, 0], P.vy + sgn * h * tv[:, 1], P.vz + sgn * h * tv[:, 2],
                             P.species_begin, P.q, P.m, P.w)
            st, G, _ = run(Pp, wl.e_tilde + sgn * h * de, wl.b_tilde + sgn * h * db)
            assert np.array_equal(st.tet, base.tet) and np.array_equal(st.n_cross, base.n_cross)
            Gs.append(G)
        fd = (Gs[0] - Gs[1]) / (2 * h)
        assert np.abs(dGt).max() > 0
        assert np.abs(fd - dGt).max() <= 1e-5 * np.abs(dGt).max(), (np.abs(fd - dGt).max(), np.abs(dGt).max())
